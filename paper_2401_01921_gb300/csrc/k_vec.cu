// FP64 vector kernels: scaling, norms and the device-resident Lanczos loop.
//
// Sec. 9.3 of arXiv 2401.01921: Lanczos needs only the operator's action on a
// vector (a LinOp).  Everything except that action runs here, in FP64, with
// no host round trip inside the loop (so a whole solve can be captured in one
// CUDA graph):
//   alpha_j = <v_j, w>;  w -= alpha_j v_j + beta_j v_{j-1};
//   twice: c = V^T w, w -= V c   (classical Gram-Schmidt, full reorthogonalisation);
//   beta_{j+1} = ||w||; stop if beta_{j+1} < 1e-14 max|alpha|; v_{j+1} = w / beta_{j+1};
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

__global__ void scale_kernel(double* x, int64_t n, double a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= a;
}

__global__ void add_scalar_kernel(double* x, int64_t n, double a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += a;
}

// partial[b] = sum over this block's grid-stride share of x*y
__global__ void __launch_bounds__(RT) dot_partial_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                                         int64_t n, double* partial, const int32_t* state) {
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
  __shared__ double sh[32];
  if (state && stopped(state)) return;
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += RT) acc += partial[i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = mode ? sqrt(acc) : acc;
}

// ---------------------------------------------------------------- Lanczos
__global__ void lanczos_init_kernel(LanczosDev L, const double* v0) {
  // V[0] = v0 / ||v0|| (norm already in L.scratch[0]); state reset
  const double inv = 1.0 / L.scratch[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += (int64_t)gridDim.x * blockDim.x)
    L.V[i] = v0[i] * inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    L.state[0] = 0;
    L.state[1] = 0;
    L.beta[0] = 0.0;
  }
}

__global__ void set_slot_kernel(double** slot, double* p) { *slot = p; }

// w -= a * v_j + b * v_{j-1}
__global__ void lanczos_axpy2_kernel(LanczosDev L, int j) {
  if (stopped(L.state)) return;
  const double a = L.alpha[j];
  const double b = L.beta[j];
  const double* vj = L.V + (int64_t)j * L.n;
  const double* vm = j > 0 ? L.V + (int64_t)(j - 1) * L.n : nullptr;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += (int64_t)gridDim.x * blockDim.x) {
    double w = L.w[i] - a * vj[i];
    if (vm) w -= b * vm[i];
    L.w[i] = w;
  }
}

// partial[b*(m) + i] = <V_i, w> over this block's contiguous chunk, i < m
__global__ void __launch_bounds__(RT) multidot_kernel(LanczosDev L, int m) {
  __shared__ double sh[32];
  if (stopped(L.state)) return;
  const int64_t chunk = (L.n + gridDim.x - 1) / gridDim.x;
  const int64_t c0 = chunk * blockIdx.x, c1 = min(L.n, c0 + chunk);
  for (int i = 0; i < m; ++i) {
    const double* v = L.V + (int64_t)i * L.n;
    double acc = 0.0;
    for (int64_t x = c0 + threadIdx.x; x < c1; x += RT) acc = fma(v[x], L.w[x], acc);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) L.partial[(int64_t)blockIdx.x * m + i] = acc;
  }
}

// coef[i] = sum_b partial[b*m + i]   (one block per i, fixed order)
__global__ void __launch_bounds__(RT) multidot_finalize_kernel(LanczosDev L, int m, int nb) {
  __shared__ double sh[32];
  if (stopped(L.state)) return;
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += RT) acc += L.partial[(int64_t)b * m + i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) L.coef[i] = acc;
}

// w -= sum_i coef[i] V_i
__global__ void __launch_bounds__(RT) gs_update_kernel(LanczosDev L, int m) {
  __shared__ double c[512];
  if (stopped(L.state)) return;
  for (int i = threadIdx.x; i < m; i += RT) c[i] = L.coef[i];
  __syncthreads();
  for (int64_t x = (int64_t)blockIdx.x * RT + threadIdx.x; x < L.n; x += (int64_t)gridDim.x * RT) {
    double w = L.w[x];
    for (int i = 0; i < m; ++i) w -= c[i] * L.V[(int64_t)i * L.n + x];
    L.w[x] = w;
  }
}

// beta_{j+1} already in L.beta[j+1]: decide stop, record k
__global__ void lanczos_decide_kernel(LanczosDev L, int j, int last) {
  if (stopped(L.state)) return;
  double amax = 0.0;
  for (int i = 0; i <= j; ++i) amax = fmax(amax, fabs(L.alpha[i]));
  L.state[0] = j + 1;
  if (last || L.beta[j + 1] < 1e-14 * amax) L.state[1] = 1;
}

__global__ void lanczos_normalize_kernel(LanczosDev L, int j) {
  if (stopped(L.state)) return;
  const double inv = 1.0 / L.beta[j + 1];
  double* vn = L.V + (int64_t)(j + 1) * L.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += (int64_t)gridDim.x * blockDim.x)
    vn[i] = L.w[i] * inv;
}

__device__ int sturm_count(const double* a, const double* b, int k, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int j = 0; j < k; ++j) {
    d = (a[j] - x) - (j > 0 ? (b[j] * b[j]) / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0) ++cnt;
  }
  return cnt;
}

// Sturm bisection for the lowest eigenvalue of T, inverse iteration for y.
// beta[j] couples rows j-1 and j (beta[0] unused).  Single thread: k is small.
__global__ void tridiag_kernel(LanczosDev L) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = L.state[0];
  const double* a = L.alpha;
  const double* b = L.beta;
  double lo = 0.0, hi = 0.0;
  for (int j = 0; j < k; ++j) {
    const double r = (j > 0 ? fabs(b[j]) : 0.0) + (j + 1 < k ? fabs(b[j + 1]) : 0.0);
    if (j == 0 || a[j] - r < lo) lo = a[j] - r;
    if (j == 0 || a[j] + r > hi) hi = a[j] + r;
  }
  for (int it = 0; it < 2000; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(a, b, k, mid) >= 1) hi = mid; else lo = mid;
  }
  const double lam = hi;
  *L.eval = lam;
  // inverse iteration (Thomas algorithm), 3 sweeps, from the normalised ones vector
  double* y = L.y;
  double* dd = L.scratch;          // k
  double* rhs = L.scratch + L.nmax; // k
  const double shift = lam - 1e-13 * fmax(1.0, fabs(lam));
  for (int j = 0; j < k; ++j) y[j] = 1.0 / sqrt((double)k);
  for (int sweep = 0; sweep < 3; ++sweep) {
    for (int j = 0; j < k; ++j) { dd[j] = a[j] - shift; rhs[j] = y[j]; }
    for (int j = 1; j < k; ++j) {
      const double piv = dd[j - 1] != 0.0 ? dd[j - 1] : 1e-300;
      const double m = b[j] / piv;
      dd[j] -= m * b[j];
      rhs[j] -= m * rhs[j - 1];
    }
    y[k - 1] = rhs[k - 1] / (dd[k - 1] != 0.0 ? dd[k - 1] : 1e-300);
    for (int j = k - 2; j >= 0; --j) y[j] = (rhs[j] - b[j + 1] * y[j + 1]) / (dd[j] != 0.0 ? dd[j] : 1e-300);
    double nrm = 0.0;
    for (int j = 0; j < k; ++j) nrm += y[j] * y[j];
    nrm = sqrt(nrm);
    for (int j = 0; j < k; ++j) y[j] /= nrm;
  }
  int jm = 0;
  for (int j = 1; j < k; ++j)
    if (fabs(y[j]) > fabs(y[jm])) jm = j;
  if (y[jm] < 0)
    for (int j = 0; j < k; ++j) y[j] = -y[j];
}

__global__ void __launch_bounds__(RT) ritz_kernel(LanczosDev L, double* out) {
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
  scale_kernel<<<grid_for(n), RT, 0, st>>>(x, n, alpha);
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_add_scalar(double* x, int64_t n, double alpha, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  add_scalar_kernel<<<grid_for(n), RT, 0, st>>>(x, n, alpha);
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_norm2(const double* x, int64_t n, double* partial, double* out, cudaStream_t st) {
  const int nb = grid_for(n);
  dot_partial_kernel<<<nb, RT, 0, st>>>(x, x, n, partial, nullptr);
  tnx_note_launch(1);
  finalize_kernel<<<1, RT, 0, st>>>(partial, nb, out, 1, nullptr);
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_lanczos_init(const LanczosDev& L, const double* v0, cudaStream_t st) {
  const int nb = grid_for(L.n);
  dot_partial_kernel<<<nb, RT, 0, st>>>(v0, v0, L.n, L.partial, nullptr);
  tnx_note_launch(1);
  finalize_kernel<<<1, RT, 0, st>>>(L.partial, nb, L.scratch, 1, nullptr);
  tnx_note_launch(1);
  lanczos_init_kernel<<<nb, RT, 0, st>>>(L, v0);
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_lanczos_set_input(double** slot_ptr, const LanczosDev& L, int j, cudaStream_t st) {
  set_slot_kernel<<<1, 1, 0, st>>>(slot_ptr, L.V + (int64_t)j * L.n);
  tnx_note_launch(1);
  return cudaGetLastError();
}

// The operator has been applied: L.w = H v_j.  One Lanczos step.
cudaError_t tnx_launch_lanczos_step(const LanczosDev& L, int j, cudaStream_t st) {
  const int nb = grid_for(L.n);
  const double* vj = L.V + (int64_t)j * L.n;
  dot_partial_kernel<<<nb, RT, 0, st>>>(vj, L.w, L.n, L.partial, L.state);
  tnx_note_launch(1);
  finalize_kernel<<<1, RT, 0, st>>>(L.partial, nb, L.alpha + j, 0, L.state);
  tnx_note_launch(1);
  lanczos_axpy2_kernel<<<nb, RT, 0, st>>>(L, j);
  tnx_note_launch(1);
  const int m = j + 1;
  for (int pass = 0; pass < 2; ++pass) {
    multidot_kernel<<<L.nblocks, RT, 0, st>>>(L, m);
    tnx_note_launch(1);
    multidot_finalize_kernel<<<m, RT, 0, st>>>(L, m, L.nblocks);
    tnx_note_launch(1);
    gs_update_kernel<<<nb, RT, 0, st>>>(L, m);
    tnx_note_launch(1);
  }
  dot_partial_kernel<<<nb, RT, 0, st>>>(L.w, L.w, L.n, L.partial, L.state);
  tnx_note_launch(1);
  finalize_kernel<<<1, RT, 0, st>>>(L.partial, nb, L.beta + j + 1, 1, L.state);
  tnx_note_launch(1);
  lanczos_decide_kernel<<<1, 1, 0, st>>>(L, j, j == L.nmax - 1);
  tnx_note_launch(1);
  lanczos_normalize_kernel<<<nb, RT, 0, st>>>(L, j);
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_lanczos_finish(const LanczosDev& L, double* evec, cudaStream_t st) {
  tridiag_kernel<<<1, 1, 0, st>>>(L);
  tnx_note_launch(1);
  if (evec) {
    ritz_kernel<<<grid_for(L.n), RT, 0, st>>>(L, evec);
    tnx_note_launch(1);
  }
  return cudaGetLastError();
}
