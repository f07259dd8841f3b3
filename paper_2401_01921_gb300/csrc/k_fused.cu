// Fused skinny contraction step: gather, FP64 product, scatter in one kernel.
//
// A contraction whose charge groups all have K <= 16 (the MPO step of the
// two-site H_eff, Sec. 11) is a small FP64 product between two relayouts: its
// operand A is gathered from the previous step's output blocks into the packed
// K-major matrix, and its output C is immediately relaid into the next step's
// packed operand.  Here one CTA takes a tile of up to 128 rows (p, q) of one row
// block of A_g:
//   1. every A element of the tile is read from its source block through the
//      descriptor of its column (consecutive threads take consecutive q, the
//      source blocks' contiguous leg), into the A rows in shared memory;
//   2. the CTA lists the nonzeros of every column of the packed B_g (the MPO
//      product is mostly zeros) and two threads form each output row (even and
//      odd columns), with the same FMA chains as the unfused skinny kernel
//      (bit-identical; a power-of-two first coefficient is applied on the
//      integer units, tnx_first_term);
//   3. every output element is stored through the descriptor of its column
//      straight into the next step's packed operand (consecutive threads take
//      consecutive p, that operand's contiguous leg), or the rows are written to
//      C_g when no next step reads them through descriptors.
// The packed A and the C rows never reach HBM when both ends are fused.  The
// descriptors are precomputed by the planner from the two relayouts' bands.
#include "tnx_internal.h"

namespace {

constexpr int FR = TNX_FUSED_ROWS; // a tile has FR rows at most, two threads per row
constexpr int FT = 2 * FR;         // threads
constexpr int FMAXN = 64;         // output columns (rows of B_g) at most
constexpr int FMAXK = 16;         // columns of A (ldK) at most
// the prologue's thread ranges: B nonzeros by threads [FR, FR + N), output
// column descriptors by [FR + FMAXN, FR + FMAXN + N), N <= FMAXN
static_assert(FR + 2 * FMAXN <= FT, "the fused tile needs FR >= 2 * FMAXN rows (threads for its prologue loads)");
static_assert((FR & (FR - 1)) == 0, "the fused tile row count must be a power of two");

struct FusedSmem {
  double s_v[FMAXN][FMAXK];       // nonzero B entries of each output column
  FusedCol s_sc[FMAXN];           // output column descriptors
  unsigned char s_k[FMAXN][FMAXK];
  int s_cnt[FMAXN];
  uint32_t s_p2[FMAXN];           // tnx_pow2_code of each column's first nonzero
};

__global__ void __launch_bounds__(FT, 6) fused_skinny_kernel(const GemmGroup* __restrict__ groups,
                                                          const FusedTile* __restrict__ tiles,
                                                          const FusedCol* __restrict__ cols, int kp, int np,
                                                          double* const* __restrict__ slots) {
  tnx_grid_dependency();
  extern __shared__ __align__(16) unsigned char dyn[];
  FusedSmem& S = *(FusedSmem*)dyn;
  double* sA = (double*)(dyn + sizeof(FusedSmem));   // [rows][kp]
  double* sC = sA + FR * kp;                         // [rows][np]
  const FusedTile T = tiles[blockIdx.x];
  const int tid = threadIdx.x, half = tid / FR, t = tid & (FR - 1);
  const int rows = T.tP * T.tQ, W = T.W, N = T.N;
  // output column descriptors (threads [FR + FMAXN, FR + FMAXN + N)), off the gather's path
  if (tid >= FR + FMAXN && tid - FR - FMAXN < N && T.scol >= 0) S.s_sc[tid - FR - FMAXN] = cols[T.scol + tid - FR - FMAXN];
  // B nonzeros (threads [FR, FR + N))
  const GemmGroup g = groups[T.group];
  if (half == 1 && t < N) {
    const int K = g.K;
    const double* brow = slots[g.b_slot] + g.b_off + (int64_t)t * g.ldb;
    double b[FMAXK];
#pragma unroll
    for (int k = 0; k < FMAXK; ++k) b[k] = k < K ? brow[k] : 0.0;
    int c = 0;
#pragma unroll
    for (int k = 0; k < FMAXK; ++k) {
      if (b[k] != 0.0) {
        S.s_v[t][c] = b[k];
        S.s_k[t][c] = (unsigned char)k;
        ++c;
      }
    }
    S.s_cnt[t] = c;
    S.s_p2[t] = c ? tnx_pow2_code(S.s_v[t][0]) : 0u;
  }
  // gather: row r = t, q fastest; this thread takes columns half, half + 2, ...
  if (t < rows) {
    const int p = t / T.tQ, q = t - p * T.tQ;
    const int64_t P = T.p0 + p, Q = T.q0 + q;
    double v[FMAXK / 2];
#pragma unroll
    for (int j = 0; j < FMAXK / 2; ++j) {
      const int c = half + 2 * j;
      v[j] = 0.0;
      if (c < W) {
        const FusedCol d = cols[T.gcol + c];
        if (d.ptr) v[j] = __ldg(d.ptr + P * d.sP + Q * d.sQ);
      }
    }
#pragma unroll
    for (int j = 0; j < FMAXK / 2; ++j) {
      const int c = half + 2 * j;
      if (c < W) sA[t * kp + c] = v[j];
    }
  }
  __syncthreads();
  if (t < rows) {
    const double* arow = sA + t * kp;
    double* crow = sC + t * np;
    for (int n = half; n < N; n += 2) {
      double acc = 0.0;
      const int c = S.s_cnt[n];
      if (c > 0) acc = tnx_first_term(arow[S.s_k[n][0]], S.s_v[n][0], S.s_p2[n]);
      for (int e = 1; e < c; ++e) acc = fma(arow[S.s_k[n][e]], S.s_v[n][e], acc);
      crow[n] = acc;
    }
  }
  __syncthreads();
  if (T.scol >= 0) {
    // scatter: p fastest (row r = p * tQ + q in shared memory)
    if (t < rows) {
      const int q = t / T.tP, p = t - q * T.tP;
      const int64_t P = T.p0 + p, Q = T.q0 + q;
      const double* crow = sC + (p * T.tQ + q) * np;
      for (int c = half; c < N; c += 2) {
        const FusedCol d = S.s_sc[c];
        if (d.ptr) d.ptr[P * d.sP + Q * d.sQ] = crow[c];
      }
    }
  } else {
    // rows (p, q) of the block are rows row0 + (p0 + p) * EQ + q0 + q of C_g,
    // EQ = the band's extent of q (the tiles of a band share T.row0 and EQ)
    double* C = slots[g.c_slot] + g.c_off;
    const int EQ = -T.scol - 1;
    for (int e = tid; e < rows * N; e += FT) {
      const int r = e / N, n = e - r * N;
      const int p = r / T.tQ, q = r - p * T.tQ;
      const int64_t row = (int64_t)T.row0 + (int64_t)(T.p0 + p) * EQ + T.q0 + q;
      C[row * g.ldc + n] = sC[r * np + n];
    }
  }
}

}  // namespace

size_t tnx_fused_smem_bytes(int kp, int np) { return sizeof(FusedSmem) + (size_t)FR * (kp + np) * sizeof(double); }

cudaError_t tnx_launch_fused_skinny(const GemmGroup* groups, const FusedTile* tiles, int ntiles, const FusedCol* cols,
                                    int kp, int np, double* const* slots, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (kp < 1 || kp > FMAXK + 1 || np < 1 || np > FMAXN + 1) return cudaErrorInvalidValue;
  const size_t smem = tnx_fused_smem_bytes(kp, np);
  static int attr_dev = -1;   // the opt-in is per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_dev != dev) {
    e = cudaFuncSetAttribute(fused_skinny_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tnx_fused_smem_bytes(FMAXK + 1, FMAXN + 1));
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  {
    const cudaError_t le =
        tnx_launch(fused_skinny_kernel, dim3(ntiles), dim3(FT), smem, st, groups, tiles, cols, kp, np, slots);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  return cudaGetLastError();
}
