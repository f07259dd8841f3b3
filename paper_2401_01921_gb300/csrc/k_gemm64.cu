// Grouped dense products for the fused charge sectors, native FP64.
//
// Sec. 7 / Sec. 10 of arXiv 2401.01921: after matching, each charge sector of
// a pairwise contraction is one dense matrix product (the paper hands these to
// BLAS / cuBLAS).  Here one launch covers every tile of every group:
// C_g[M,N] = A_g[M,K] * B_g[N,K]^T, operands K-major, C row-major.
//
// 64x64 output tile per CTA of 256 threads, each thread a 4x4 register tile
// of FP64 FMAs; K staged through shared memory in slices of 16.  FP64 on this
// part runs at a small fraction of its FP32 / tensor rate, so the kernel is
// bound by the FP64 pipe, not by memory; ragged tile edges are masked.
// The FP32 variant (operands rounded to FP32, FP32 FMAs, result widened) is
// the "single FP32" point of the precision sweep.
#include "tnx_internal.h"

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <typename TC>
__global__ void __launch_bounds__(256) gemm_kernel(const GemmGroup* __restrict__ groups,
                                                   const GemmTile* __restrict__ tiles,
                                                   double* const* __restrict__ slots) {
  tnx_grid_dependency();
  __shared__ TC As[BK][BM + 1];
  __shared__ TC Bs[BK][BN + 1];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmGroup g = groups[tl.group];
  const double* A = slots[g.a_slot] + g.a_off;
  const double* B = slots[g.b_slot] + g.b_off;
  double* C = slots[g.c_slot] + g.c_off;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  TC acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    // load 64x16 of A and of B (1024 elements each, 4 per thread), k fastest
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = threadIdx.x + r * 256;
      const int row = idx >> 4, kk = idx & 15;
      const int gm = tl.m0 + row, gn = tl.n0 + row, gk = k0 + kk;
      As[kk][row] = (gm < g.M && gk < g.K) ? (TC)A[(int64_t)gm * g.lda + gk] : (TC)0;
      Bs[kk][row] = (gn < g.N && gk < g.K) ? (TC)B[(int64_t)gn * g.ldb + gk] : (TC)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TC a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = tl.m0 + ty + 16 * i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = tl.n0 + tx + 16 * j;
      if (gn < g.N) C[(int64_t)gm * g.ldc + gn] = (double)acc[i][j];
    }
  }
}

// Skinny products (K <= 16): one thread per row of a 128 x 64 tile.  The
// MPO-like operand B of these steps is small and mostly zeros (the two-site
// MPO product of the Heisenberg H_eff stores 30 nonzeros in 114 entries), and
// FP64 FMAs are the scarce resource of this part: each CTA first lists the
// nonzeros of every output column of its tile in shared memory (one thread per
// column, in k order), then every thread walks those lists against its row of
// A (staged in shared memory).  Skipping a zero term leaves an FMA chain
// unchanged, so the result equals the dense product bit for bit.
constexpr int SK_MAXK = 16;

__global__ void __launch_bounds__(128) gemm_skinny_kernel(const GemmGroup* __restrict__ groups,
                                                          const GemmTile* __restrict__ tiles,
                                                          double* const* __restrict__ slots) {
  tnx_grid_dependency();
  __shared__ double s_v[64][SK_MAXK];          // nonzero B entries of each output column
  __shared__ unsigned char s_k[64][SK_MAXK];   // their k
  __shared__ int s_cnt[64];
  __shared__ uint32_t s_p2[64];                // tnx_pow2_code of the first nonzero
  __shared__ double s_a[128][SK_MAXK + 1];     // the CTA's rows of A (padded: conflict-free)
  const GemmTile tl = tiles[blockIdx.x];
  const GemmGroup g = groups[tl.group];
  const double* A = slots[g.a_slot] + g.a_off;
  const double* B = slots[g.b_slot] + g.b_off;
  double* C = slots[g.c_slot] + g.c_off;
  const int nn = min(64, g.N - tl.n0);
  const int K = g.K;
  if ((int)threadIdx.x < nn) {
    const double* brow = B + (int64_t)(tl.n0 + threadIdx.x) * g.ldb;
    int c = 0;
    for (int k = 0; k < K; ++k) {
      const double v = brow[k];
      if (v != 0.0) {
        s_v[threadIdx.x][c] = v;
        s_k[threadIdx.x][c] = (unsigned char)k;
        ++c;
      }
    }
    s_cnt[threadIdx.x] = c;
    s_p2[threadIdx.x] = c ? tnx_pow2_code(s_v[threadIdx.x][0]) : 0u;
  }
  const int m = tl.m0 + threadIdx.x;
  if (m < g.M) {
    double a[SK_MAXK];
#pragma unroll
    for (int k = 0; k < SK_MAXK; ++k)
      if (k < K) a[k] = A[(int64_t)m * g.lda + k];
#pragma unroll
    for (int k = 0; k < SK_MAXK; ++k)
      if (k < K) s_a[threadIdx.x][k] = a[k];
  }
  __syncthreads();
  if (m >= g.M) return;
  const double* arow = s_a[threadIdx.x];
  double* crow = C + (int64_t)m * g.ldc + tl.n0;
  for (int n = 0; n < nn; ++n) {
    double acc = 0.0;
    const int c = s_cnt[n];
    if (c > 0) acc = tnx_first_term(arow[s_k[n][0]], s_v[n][0], s_p2[n]);
    for (int e = 1; e < c; ++e) acc = fma(arow[s_k[n][e]], s_v[n][e], acc);
    crow[n] = acc;
  }
}

}  // namespace

cudaError_t tnx_launch_gemm_skinny(const GemmGroup* groups, const GemmTile* tiles, int ntiles, double* const* slots,
                                   cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  {
    const cudaError_t le = tnx_launch(gemm_skinny_kernel, dim3(ntiles), dim3(128), 0, st, groups, tiles, slots);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_gemm_f64(const GemmGroup* groups, const GemmTile* tiles, int ntiles,
                                double* const* slots, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  {
    const cudaError_t le = tnx_launch(gemm_kernel<double>, dim3(ntiles), dim3(256), 0, st, groups, tiles, slots);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_gemm_f32(const GemmGroup* groups, const GemmTile* tiles, int ntiles,
                                double* const* slots, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  {
    const cudaError_t le = tnx_launch(gemm_kernel<float>, dim3(ntiles), dim3(256), 0, st, groups, tiles, slots);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  return cudaGetLastError();
}
