// FP64 vector kernels: scaling, norms and the device-resident Lanczos loop.
//
// Sec. 9.3 of arXiv 2401.01921: Lanczos needs only the operator's action on a
// vector (a LinOp).  Everything except that action runs here, in FP64, with
// no host round trip inside the loop (so a whole solve can be captured in one
// CUDA graph):
//   alpha_j = <v_j, w>; w -= alpha_j v_j + beta_j v_{j-1} (three-term step);
//   c = V^T w, w -= V c   (one classical Gram-Schmidt pass against every
//   previous vector: full reorthogonalisation);
//   beta_{j+1} = ||w||; stop if beta_{j+1} < 1e-14 max(|alpha_i|, beta_i; i <= j);
//   v_{j+1} = w / beta_{j+1};
// then Sturm bisection on the tridiagonal T and inverse iteration for its
// eigenvector, and the Ritz vector V y.
// Reductions are deterministic: per-block partial sums with a fixed grid and
// a fixed-order tree (warp shuffles), then one block summing the partials in
// a fixed order.
#include "tnx_internal.h"

namespace {

constexpr int RT = 256;        // threads per reduction block
constexpr int RBLOCKS = 1216;  // 8 blocks per SM on 152 SMs

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum, result valid in thread 0
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}

__device__ __forceinline__ bool stopped(const int32_t* state) { return *(volatile const int32_t*)(state + 1) != 0; }

// A gated launch of the Gram-Schmidt pass does nothing unless this step's
// decision asked for the pass.
__device__ __forceinline__ bool gated_off(const int32_t* state, int gate) {
  return gate && *(volatile const int32_t*)(state + 2) == 0;
}

// Reductions finish in the launch that produces their partial sums: every
// block publishes its partials, fences and counts itself in state[4]; the
// block that counts last (no block waits for another) reads all partials
// through L2, in a fixed order, so the result does not depend on which block
// that is, and resets the counter for the next launch.
__device__ bool last_block(int32_t* counter) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(counter, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

__global__ void scale_kernel(double* x, int64_t n, double a) {
  tnx_grid_dependency();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= a;
}

__global__ void add_scalar_kernel(double* x, int64_t n, double a) {
  tnx_grid_dependency();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += a;
}

// partial[b] = sum over this block's grid-stride share of x*y
__global__ void __launch_bounds__(RT) dot_partial_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                                         int64_t n, double* partial, const int32_t* state) {
  tnx_grid_dependency();
  __shared__ double sh[32];
  if (state && stopped(state)) return;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * RT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RT)
    acc = fma(x[i], y[i], acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// mode 0: out = sum; mode 1: out = sqrt(sum)
__global__ void __launch_bounds__(RT) finalize_kernel(const double* partial, int np, double* out, int mode,
                                                      const int32_t* state) {
  tnx_grid_dependency();
  __shared__ double sh[32];
  if (state && stopped(state)) return;
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += RT) acc += partial[i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = mode ? sqrt(acc) : acc;
}

// ---------------------------------------------------------------- Lanczos
__global__ void lanczos_init_kernel(LanczosDev L, const double* v0) {
  tnx_grid_dependency();
  // V[0] = v0 / ||v0|| (norm already in L.scratch[0]); state reset
  const double inv = 1.0 / L.scratch[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += (int64_t)gridDim.x * blockDim.x)
    L.V[i] = v0[i] * inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    L.state[0] = 0;
    L.state[1] = 0;
    L.state[2] = 0;
    L.state[3] = 0;
    L.state[4] = 0;   // the last-block counter
    L.beta[0] = 0.0;
    L.omega[0] = 1.0;   // <v_0, v_0>; the row before it is empty
  }
}

__global__ void set_slot_kernel(double** slot, double* p) {
  tnx_grid_dependency();
  *slot = p;
}

// partial[b*m + i] = <V_i, w> over this block's contiguous chunk, i < m.  A
// grid of multidot_blocks(n) blocks keeps the number of partial sums (and so the
// FP64 additions of the reduction tree) bounded; each thread keeps NG <= 16
// running sums (NG fixed at compile time, so no FP64 instruction is issued for
// a vector that does not exist), w is read once per group of vectors, and the
// block reduction goes through shared memory: 16 rows of MD_T values, 8
// threads per row.  FP64 issue slots are scarce on this part, so the grid is
// only large enough to keep the loads in flight.
constexpr int MD_T = 128;
constexpr int MD_BLOCKS_MAX = 608;

// Blocks of the multidot kernel: about 416 vector entries per block (an
// L2-resident basis is bound by FP64 issue, where fewer partial sums help),
// rounded to a multiple of the SM count, at least 1 and at most 4 per SM (a
// basis in HBM needs the loads of that many blocks in flight).
int multidot_blocks(int64_t n) {
  int64_t b = (n / 416 + 151) / 152 * 152;
  if (b < 152) b = 152;
  if (b > MD_BLOCKS_MAX) b = MD_BLOCKS_MAX;
  return (int)b;
}

template <int NG>
__device__ __forceinline__ void multidot_group(const LanczosDev& L, int g0, int64_t c0, int64_t c1,
                                               double (*sh)[MD_T + 1]) {
  // g0 is the basis row of the group's first vector
  double acc[NG];
#pragma unroll
  for (int i = 0; i < NG; ++i) acc[i] = 0.0;
  // two entries per iteration: both rows' loads are in flight before the FMAs
  int64_t x = c0 + threadIdx.x;
  for (; x + MD_T < c1; x += 2 * MD_T) {
    const double w0 = L.w[x], w1 = L.w[x + MD_T];
    double v0[NG], v1[NG];
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      v0[i] = L.V[(int64_t)(g0 + i) * L.n + x];
      v1[i] = L.V[(int64_t)(g0 + i) * L.n + x + MD_T];
    }
#pragma unroll
    for (int i = 0; i < NG; ++i) acc[i] = fma(v1[i], w1, fma(v0[i], w0, acc[i]));
  }
  if (x < c1) {
    const double wx = L.w[x];
#pragma unroll
    for (int i = 0; i < NG; ++i) acc[i] = fma(L.V[(int64_t)(g0 + i) * L.n + x], wx, acc[i]);
  }
#pragma unroll
  for (int i = 0; i < NG; ++i) sh[i][threadIdx.x] = acc[i];
}

// Dots of this block's chunk [c0, c1) against V_vb .. V_{vb+m-1} into partial[b*m + i].
__device__ void block_multidot(const LanczosDev& L, int m, int64_t c0, int64_t c1, double (*sh)[MD_T + 1],
                               int vb = 0) {
  for (int g0 = 0; g0 < m; g0 += 16) {
    const int ng = m - g0 < 16 ? m - g0 : 16;
    const int r0 = vb + g0;
    switch (ng) {
      case 1: multidot_group<1>(L, r0, c0, c1, sh); break;
      case 2: multidot_group<2>(L, r0, c0, c1, sh); break;
      case 3: multidot_group<3>(L, r0, c0, c1, sh); break;
      case 4: multidot_group<4>(L, r0, c0, c1, sh); break;
      case 5: multidot_group<5>(L, r0, c0, c1, sh); break;
      case 6: multidot_group<6>(L, r0, c0, c1, sh); break;
      case 7: multidot_group<7>(L, r0, c0, c1, sh); break;
      case 8: multidot_group<8>(L, r0, c0, c1, sh); break;
      case 9: multidot_group<9>(L, r0, c0, c1, sh); break;
      case 10: multidot_group<10>(L, r0, c0, c1, sh); break;
      case 11: multidot_group<11>(L, r0, c0, c1, sh); break;
      case 12: multidot_group<12>(L, r0, c0, c1, sh); break;
      case 13: multidot_group<13>(L, r0, c0, c1, sh); break;
      case 14: multidot_group<14>(L, r0, c0, c1, sh); break;
      case 15: multidot_group<15>(L, r0, c0, c1, sh); break;
      default: multidot_group<16>(L, r0, c0, c1, sh); break;
    }
    __syncthreads();
    // thread t sums 16 consecutive entries of row t/8, then 8 partners combine
    const int row = threadIdx.x >> 3, part = threadIdx.x & 7;
    if (row < ng) {
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < MD_T / 8; ++q) v += sh[row][part * (MD_T / 8) + q];
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) v += __shfl_down_sync(0xffu << (threadIdx.x & 24), v, o, 8);
      if (part == 0) L.partial[(int64_t)blockIdx.x * m + g0 + row] = v;
    }
    __syncthreads();
  }
}

// coef[i] = sum_b partial[b*m + i] over the nb blocks of the launch (fixed
// order); the sum of row alpha_i (if >= 0) is also alpha_j = <v_j, H v_j>.
// Run by one block of any width.
__device__ void finalize_coefs(const LanczosDev& L, int m, int nb, int alpha_i, int alpha_j, double* sh) {
  for (int i = 0; i < m; ++i) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += __ldcg(L.partial + (int64_t)b * m + i);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) {
      L.coef[i] = acc;
      if (i == alpha_i) L.alpha[alpha_j] = acc;
    }
  }
}

// Dots of w against V_vb .. V_{vb+m-1}, the coefficients formed by the last block.
__global__ void __launch_bounds__(MD_T) multidot_kernel(LanczosDev L, int m, int vb, int gate, int alpha_i,
                                                        int alpha_j) {
  tnx_grid_dependency();
  __shared__ double sh[16][MD_T + 1];
  __shared__ double shr[32];
  if (stopped(L.state) || gated_off(L.state, gate)) return;
  const int64_t chunk = (L.n + gridDim.x - 1) / gridDim.x;
  const int64_t c0 = chunk * blockIdx.x, c1 = min(L.n, c0 + chunk);
  block_multidot(L, m, c0, c1, sh, vb);
  if (last_block(L.state + 4)) {
    finalize_coefs(L, m, gridDim.x, alpha_i, alpha_j, shr);
    if (threadIdx.x == 0) L.state[4] = 0;
  }
}

// beta_{j+1} = sqrt(sum of the nb norm partials); decide stop; record k; point
// the next apply's input slot at v_{j+1} (which the next kernel writes).  Run
// by one block of RT threads.
__device__ void beta_decide(const LanczosDev& L, int j, int nb, int last, double** next_slot) {
  __shared__ double sh[32];
  __shared__ double s_amax;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += RT) acc += __ldcg(L.partial + b);
  if (threadIdx.x < 32) {
    double amax = 0.0;
    // the scale of T seen so far: max |alpha_i| and max beta_i (i <= j; beta_0 = 0)
    for (int i = threadIdx.x; i <= j; i += 32) amax = fmax(amax, fmax(fabs(L.alpha[i]), L.beta[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (threadIdx.x == 0) s_amax = amax;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    const double beta = sqrt(acc);
    L.beta[j + 1] = beta;
    L.scratch[3 * L.nmax + 3] = 1.0 / beta;   // for the normalising kernel
    L.state[0] = j + 1;
    if (last || beta < 1e-14 * s_amax) L.state[1] = 1;
    else *next_slot = L.V + (int64_t)(j + 1) * L.n;
  }
}

// w -= sum_i coef[i] V_i; with norm != 0 also partial[b] = sum of the new w^2
// over this block's grid-stride share (fixed order).
__global__ void __launch_bounds__(RT) gs_update_kernel(LanczosDev L, int m, int norm, int gate, int j, int last,
                                                        double** next_slot) {
  tnx_grid_dependency();
  __shared__ double c[512];
  __shared__ double sh[32];
  if (stopped(L.state) || gated_off(L.state, gate)) return;
  for (int i = threadIdx.x; i < m; i += RT) c[i] = L.coef[i];
  __syncthreads();
  double nrm = 0.0;
  // two entries per iteration (the second one stride later), so that the loads
  // of both are in flight together; each entry keeps its own subtraction order
  const int64_t stride = (int64_t)gridDim.x * RT;
  int64_t x = (int64_t)blockIdx.x * RT + threadIdx.x;
  for (; x + stride < L.n; x += 2 * stride) {
    double w0 = L.w[x], w1 = L.w[x + stride];
#pragma unroll 4
    for (int i = 0; i < m; ++i) {
      const double* vi = L.V + (int64_t)i * L.n;
      const double a0 = vi[x], a1 = vi[x + stride];
      w0 -= c[i] * a0;
      w1 -= c[i] * a1;
    }
    L.w[x] = w0;
    L.w[x + stride] = w1;
    nrm = fma(w0, w0, nrm);
    nrm = fma(w1, w1, nrm);
  }
  if (x < L.n) {
    double w = L.w[x];
#pragma unroll 8
    for (int i = 0; i < m; ++i) w -= c[i] * L.V[(int64_t)i * L.n + x];
    L.w[x] = w;
    nrm = fma(w, w, nrm);
  }
  if (norm) {
    nrm = block_sum(nrm, sh);
    if (threadIdx.x == 0) L.partial[blockIdx.x] = nrm;
    // the last block: beta_{j+1} and the stopping test of this step
    if (last_block(L.state + 4)) {
      beta_decide(L, j, gridDim.x, last, next_slot);
      if (threadIdx.x == 0) L.state[4] = 0;
    }
  }
}

// Partial reorthogonalisation (Simon, Math. Comp. 42, 1984): omega_{j,k}
// estimates <v_j, v_k> through the recurrence that the Lanczos relation gives,
//   beta_{j+1} omega_{j+1,k} = beta_{k+1} omega_{j,k+1} + (alpha_k - alpha_j) omega_{j,k}
//                              + beta_k omega_{j,k-1} - beta_j omega_{j-1,k} + rounding,
// with the rounding term taken as sign(.) eps1 |T| (eps1 = sqrt(n) eps / 2, |T|
// bounded by max_i |alpha_i| + beta_i + beta_{i+1}) and omega_{j+1,j} =
// eps1 |T| / beta_{j+1}.  After the three-term step this kernel forms
// beta_{j+1} = |w| and the estimates of row j+1; the step takes a full
// Gram-Schmidt pass against v_0..v_j when the largest estimate exceeds
// tau (1e-10; a negative tau: every step), and so does the step after it (the error that v_j carries reaches
// v_{j+2} too); after a pass the estimates restart at eps1.  Without a pass
// it also does what beta_decide does (beta_{j+1}, the stopping
// test, the next input slot); with one, the gated launches after it do.
constexpr int PRO_MAX = 514;   // rows of at most 500 steps + 2

// Run by one block of RT threads over the nb norm partials.
__device__ void pro_decide(const LanczosDev& L, int j, int nb, int last, double** next_slot, double tau) {
  __shared__ double sh[32];
  __shared__ double s_om[PRO_MAX];
  __shared__ double s_b, s_amax, s_anorm, s_mx[RT / 32];
  __shared__ int s_pass;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += RT) acc += __ldcg(L.partial + b);
  if (threadIdx.x < 32) {
    double amax = 0.0, an = 0.0;
    for (int i = threadIdx.x; i <= j; i += 32) {
      amax = fmax(amax, fmax(fabs(L.alpha[i]), L.beta[i]));
      an = fmax(an, fabs(L.alpha[i]) + L.beta[i] + (i < j ? L.beta[i + 1] : 0.0));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      an = fmax(an, __shfl_xor_sync(0xffffffffu, an, o));
    }
    if (threadIdx.x == 0) {
      s_amax = amax;
      s_anorm = an;
    }
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) s_b = sqrt(acc);
  __syncthreads();
  const double bn = s_b;
  const double anorm = fmax(s_anorm, fabs(L.alpha[j]) + (j > 0 ? L.beta[j] : 0.0) + bn);
  const double eps1 = sqrt((double)L.n) * 0.5 * 2.220446049250313e-16;
  const double* om = L.omega;                  // row j: k = 0..j
  const double* omp = L.omega + (L.nmax + 2);  // row j-1: k = 0..j-1
  double mx = 0.0;
  for (int k = threadIdx.x; k <= j; k += RT) {
    double e;
    if (k < j) {
      double t = L.beta[k + 1] * om[k + 1] + (L.alpha[k] - L.alpha[j]) * om[k] - L.beta[j] * omp[k];
      if (k > 0) t += L.beta[k] * om[k - 1];
      e = (t + copysign(eps1 * anorm, t)) / bn;
    } else {
      e = eps1 * anorm / bn;
    }
    s_om[k] = e;
    // beta_{j+1} = 0 or an overflowing estimate counts as lost orthogonality
    mx = (fabs(e) <= 1e300) ? fmax(mx, fabs(e)) : INFINITY;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) s_mx[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < RT / 32; ++w) m = fmax(m, s_mx[w]);
    const int forced = L.state[3];
    const int pass = forced || !(m <= tau);
    s_pass = pass;
    L.state[2] = pass;
    L.state[3] = pass && !forced;
    if (!pass) {
      L.beta[j + 1] = bn;
      L.scratch[3 * L.nmax + 3] = 1.0 / bn;   // for the normalising kernel
      L.state[0] = j + 1;
      if (last || bn < 1e-14 * s_amax) L.state[1] = 1;
      else *next_slot = L.V + (int64_t)(j + 1) * L.n;
    }
  }
  __syncthreads();
  // shift the rows: row j becomes row j-1, the new estimates row j+1
  double* cur = L.omega;
  double* prev = L.omega + (L.nmax + 2);
  for (int k = threadIdx.x; k <= j; k += RT) {
    prev[k] = cur[k];
    cur[k] = s_pass ? eps1 : s_om[k];
  }
  if (threadIdx.x == 0) cur[j + 1] = 1.0;
}

// The three-term step w <- (w - alpha_j v_j) - beta_j v_{j-1} (beta_0 = 0), with
// partial[b] = this block's share of the new |w|^2 (fixed order).
__global__ void __launch_bounds__(RT) three_term_norm_kernel(LanczosDev L, int j, int last, double** next_slot,
                                                              double tau) {
  tnx_grid_dependency();
  __shared__ double sh[32];
  if (stopped(L.state)) return;
  const double a = L.alpha[j], b = j > 0 ? L.beta[j] : 0.0;
  const double* vj = L.V + (int64_t)j * L.n;
  const double* vp = L.V + (int64_t)(j > 0 ? j - 1 : 0) * L.n;
  double nrm = 0.0;
  const int64_t stride = (int64_t)gridDim.x * RT;
  int64_t x = (int64_t)blockIdx.x * RT + threadIdx.x;
  for (; x + stride < L.n; x += 2 * stride) {
    const double w0 = L.w[x], w1 = L.w[x + stride];
    const double a0 = vj[x], a1 = vj[x + stride];
    const double p0 = vp[x], p1 = vp[x + stride];
    const double u0 = (w0 - a * a0) - b * p0, u1 = (w1 - a * a1) - b * p1;
    L.w[x] = u0;
    L.w[x + stride] = u1;
    nrm = fma(u0, u0, nrm);
    nrm = fma(u1, u1, nrm);
  }
  if (x < L.n) {
    const double u = (L.w[x] - a * vj[x]) - b * vp[x];
    L.w[x] = u;
    nrm = fma(u, u, nrm);
  }
  nrm = block_sum(nrm, sh);
  if (threadIdx.x == 0) L.partial[blockIdx.x] = nrm;
  if (last_block(L.state + 4)) {
    pro_decide(L, j, gridDim.x, last, next_slot, tau);
    if (threadIdx.x == 0) L.state[4] = 0;
  }
}

__global__ void lanczos_normalize_kernel(LanczosDev L, int j) {
  tnx_grid_dependency();
  if (stopped(L.state)) return;
  const double inv = L.scratch[3 * L.nmax + 3];   // 1 / beta_{j+1}, one FP64 division per step
  double* vn = L.V + (int64_t)(j + 1) * L.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += (int64_t)gridDim.x * blockDim.x)
    vn[i] = L.w[i] * inv;
}

// A key that orders doubles as integers (-0 and +0 share key 0), and back.
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : (long long)(0x8000000000000000ull - (unsigned long long)b);
}
__device__ __forceinline__ double dfromkey(long long key) {
  return __longlong_as_double(key >= 0 ? key : (long long)(0x8000000000000000ull - (unsigned long long)key));
}

// Sturm count on the shared-memory copy of T: number of negative pivots of the
// LDL^T factorisation of T - xI (b2[j] = beta_j^2, b2[0] unused).
__device__ int sturm_count(const double* a, const double* b2, int k, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int j = 0; j < k; ++j) {
    d = (a[j] - x) - (j > 0 ? b2[j] / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0) ++cnt;
  }
  return cnt;
}

// Lowest eigenvalue of T by Sturm-sequence multisection: each of the RT
// threads counts the eigenvalues below its own point of the current bracket,
// and the bracket shrinks to the one sub-interval where the count first
// reaches 1 (the same test as bisection, RT points per round), until it stops
// shrinking.  Then inverse iteration (Thomas algorithm, 3 sweeps) for the
// eigenvector y on thread 0.  beta[j] couples rows j-1 and j (beta[0] unused).
// T is copied to shared memory first: the sequential parts run on thread 0,
// where every global-memory access would be a dependent trip to L2; the LU
// factors of T - shift I are the same in every sweep and computed once.
constexpr int TD_MAX = 512;   // Lanczos steps are limited to 500

__global__ void __launch_bounds__(RT) tridiag_kernel(LanczosDev L) {
  tnx_grid_dependency();
  __shared__ double sa[TD_MAX], sb[TD_MAX], sb2[TD_MAX], sl[TD_MAX], sy[TD_MAX];
  __shared__ double s_lo, s_hi;
  __shared__ int s_first;
  const int k = L.state[0];
  for (int j = threadIdx.x; j < k; j += RT) {
    sa[j] = L.alpha[j];
    sb[j] = L.beta[j];
    sb2[j] = j > 0 ? sb[j] * sb[j] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double lo = 0.0, hi = 0.0;
    for (int j = 0; j < k; ++j) {
      const double r = (j > 0 ? fabs(sb[j]) : 0.0) + (j + 1 < k ? fabs(sb[j + 1]) : 0.0);
      if (j == 0 || sa[j] - r < lo) lo = sa[j] - r;
      if (j == 0 || sa[j] + r > hi) hi = sa[j] + r;
    }
    s_lo = lo;
    s_hi = hi;
  }
  __syncthreads();
  const double frac = (double)(threadIdx.x + 1) / (double)(RT + 1);
  for (int round = 0; round < 64; ++round) {
    const double lo = s_lo, hi = s_hi;
    const double x = lo + (hi - lo) * frac;
    if (threadIdx.x == 0) s_first = RT;
    __syncthreads();
    if (x > lo && x < hi && sturm_count(sa, sb2, k, x) >= 1) atomicMin(&s_first, (int)threadIdx.x);
    __syncthreads();
    if (threadIdx.x == 0) {
      const int f = s_first;
      const double nlo = f == 0 ? lo : lo + (hi - lo) * ((double)f / (double)(RT + 1));
      const double nhi = f == RT ? hi : lo + (hi - lo) * ((double)(f + 1) / (double)(RT + 1));
      s_lo = nlo > lo ? nlo : lo;
      s_hi = nhi < hi ? nhi : hi;
    }
    __syncthreads();
    if (!(s_lo < s_hi) || (s_lo == lo && s_hi == hi)) break;
  }
  // Finish on the (tiny) bracket: the oracle bisects until lo and hi are
  // adjacent doubles, which leaves hi = the smallest double of (lo, hi] whose
  // count reaches 1.  Here the RT threads test the doubles lo+1, lo+2, ... ulps
  // at once (a key that orders doubles like integers), after serial halving
  // while more than RT of them remain.
  __shared__ int s_t;
  double lo = s_lo, hi = s_hi;
  if (threadIdx.x == 0) {
    for (int it = 0; it < 200 && dkey(hi) - dkey(lo) > RT; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (sturm_count(sa, sb2, k, mid) >= 1) hi = mid; else lo = mid;
    }
    s_lo = lo;
    s_hi = hi;
    s_t = RT;
  }
  __syncthreads();
  lo = s_lo;
  hi = s_hi;
  const long long span = dkey(hi) - dkey(lo);   // hi itself counts
  if ((long long)threadIdx.x + 1 < span) {
    const double x = dfromkey(dkey(lo) + threadIdx.x + 1);
    if (sturm_count(sa, sb2, k, x) >= 1) atomicMin(&s_t, (int)threadIdx.x);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double lam = s_t < RT ? dfromkey(dkey(lo) + s_t + 1) : hi;
  *L.eval = lam;
  // LU of T - shift I (no pivoting): sa becomes the pivots, sl the multipliers;
  // the sweeps multiply by the pivots' reciprocals, formed once
  const double shift = lam - 1e-13 * fmax(1.0, fabs(lam));
  for (int j = 0; j < k; ++j) sa[j] -= shift;
  for (int j = 1; j < k; ++j) {
    const double piv = sa[j - 1] != 0.0 ? sa[j - 1] : 1e-300;
    sl[j] = sb[j] / piv;
    sa[j] -= sl[j] * sb[j];
  }
  for (int j = 0; j < k; ++j) sb2[j] = 1.0 / (sa[j] != 0.0 ? sa[j] : 1e-300);   // sb2 is free now
  const double inv0 = 1.0 / sqrt((double)k);
  for (int j = 0; j < k; ++j) sy[j] = inv0;
  for (int sweep = 0; sweep < 3; ++sweep) {
    for (int j = 1; j < k; ++j) sy[j] -= sl[j] * sy[j - 1];
    sy[k - 1] = sy[k - 1] * sb2[k - 1];
    for (int j = k - 2; j >= 0; --j) sy[j] = (sy[j] - sb[j + 1] * sy[j + 1]) * sb2[j];
    double nrm = 0.0;
    for (int j = 0; j < k; ++j) nrm += sy[j] * sy[j];
    const double inv = 1.0 / sqrt(nrm);
    for (int j = 0; j < k; ++j) sy[j] *= inv;
  }
  int jm = 0;
  for (int j = 1; j < k; ++j)
    if (fabs(sy[j]) > fabs(sy[jm])) jm = j;
  const double sgn = sy[jm] < 0 ? -1.0 : 1.0;
  for (int j = 0; j < k; ++j) L.y[j] = sgn * sy[j];
}

__global__ void __launch_bounds__(RT) ritz_kernel(LanczosDev L, double* out) {
  tnx_grid_dependency();
  __shared__ double c[512];
  const int k = L.state[0];
  for (int i = threadIdx.x; i < k; i += RT) c[i] = L.y[i];
  __syncthreads();
  for (int64_t x = (int64_t)blockIdx.x * RT + threadIdx.x; x < L.n; x += (int64_t)gridDim.x * RT) {
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += c[i] * L.V[(int64_t)i * L.n + x];
    out[x] = s;
  }
}

int grid_for(int64_t n) {
  int64_t b = (n + RT - 1) / RT;
  return (int)(b < RBLOCKS ? (b < 1 ? 1 : b) : RBLOCKS);
}

}  // namespace

int tnx_reduce_blocks(int64_t n) { return grid_for(n); }

cudaError_t tnx_launch_scale(double* x, int64_t n, double alpha, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  {
    const cudaError_t le = tnx_launch(scale_kernel, dim3(grid_for(n)), dim3(RT), 0, st, x, n, alpha);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_add_scalar(double* x, int64_t n, double alpha, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  {
    const cudaError_t le = tnx_launch(add_scalar_kernel, dim3(grid_for(n)), dim3(RT), 0, st, x, n, alpha);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_norm2(const double* x, int64_t n, double* partial, double* out, cudaStream_t st) {
  const int nb = grid_for(n);
  {
    const cudaError_t le = tnx_launch(dot_partial_kernel, dim3(nb), dim3(RT), 0, st, x, x, n, partial, nullptr);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  {
    const cudaError_t le = tnx_launch(finalize_kernel, dim3(1), dim3(RT), 0, st, partial, nb, out, 1, nullptr);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_lanczos_init(const LanczosDev& L, const double* v0, cudaStream_t st) {
  const int nb = grid_for(L.n);
  {
    const cudaError_t le = tnx_launch(dot_partial_kernel, dim3(nb), dim3(RT), 0, st, v0, v0, L.n, L.partial, nullptr);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  {
    const cudaError_t le = tnx_launch(finalize_kernel, dim3(1), dim3(RT), 0, st,
                                      L.partial, nb, L.scratch, 1, nullptr);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  {
    const cudaError_t le = tnx_launch(lanczos_init_kernel, dim3(nb), dim3(RT), 0, st, L, v0);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_lanczos_set_input(double** slot_ptr, const LanczosDev& L, int j, cudaStream_t st) {
  {
    const cudaError_t le = tnx_launch(set_slot_kernel, dim3(1), dim3(1), 0, st, slot_ptr, L.V + (int64_t)j * L.n);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  return cudaGetLastError();
}

// The operator has been applied: L.w = H v_j.  One Lanczos step (without the
// final v_{j+1} = w / beta_{j+1} when `normalize` is false: the caller then
// fuses it with the next apply's relayout of the vector): alpha_j = <v_j, w>;
// the three-term step w <- w - alpha_j v_j - beta_j v_{j-1} with |w|; the
// orthogonality estimates, which decide whether this step takes a classical
// Gram-Schmidt pass c = V^T w, w <- w - V c against v_0..v_j (the gated
// launches: a step without the pass returns from them at once); then
// beta_{j+1}, the stopping test and v_{j+1} = w / beta_{j+1}.  FP64 work per
// entry: 3 fused multiply-adds, plus 2 (j + 1) + 1 in a step with the pass.
cudaError_t tnx_launch_lanczos_step(const LanczosDev& L, int j, double** next_slot, cudaStream_t st, bool normalize,
                                    bool always_pass) {
  if (j + 2 > PRO_MAX) return cudaErrorInvalidValue;
  const double tau = always_pass ? -1.0 : 1e-10;
  const int nb = grid_for(L.n);
  const int m = j + 1;
  const int mb = multidot_blocks(L.n);
  const int last = j == L.nmax - 1;
  {
    const cudaError_t le = tnx_launch(multidot_kernel, dim3(mb), dim3(MD_T), 0, st, L, 1, j, 0, 0, j);
    if (le != cudaSuccess) return le;
  }
  {
    const cudaError_t le = tnx_launch(three_term_norm_kernel, dim3(nb), dim3(RT), 0, st, L, j, last, next_slot, tau);
    if (le != cudaSuccess) return le;
  }
  {
    const cudaError_t le = tnx_launch(multidot_kernel, dim3(mb), dim3(MD_T), 0, st, L, m, 0, 1, -1, 0);
    if (le != cudaSuccess) return le;
  }
  {
    const cudaError_t le = tnx_launch(gs_update_kernel, dim3(nb), dim3(RT), 0, st, L, m, 1, 1, j, last, next_slot);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(4);
  if (normalize) {
    {
      const cudaError_t le = tnx_launch(lanczos_normalize_kernel, dim3(nb), dim3(RT), 0, st, L, j);
      if (le != cudaSuccess) return le;
    }
    tnx_note_launch(1);
  }
  return cudaGetLastError();
}

cudaError_t tnx_launch_lanczos_finish(const LanczosDev& L, double* evec, cudaStream_t st) {
  {
    const cudaError_t le = tnx_launch(tridiag_kernel, dim3(1), dim3(RT), 0, st, L);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  if (evec) {
    {
      const cudaError_t le = tnx_launch(ritz_kernel, dim3(grid_for(L.n)), dim3(RT), 0, st, L, evec);
      if (le != cudaSuccess) return le;
    }
    tnx_note_launch(1);
  }
  return cudaGetLastError();
}
