// Singular value decomposition of the dense charge blocks of a block-sparse
// tensor (Sec. 9.2 of arXiv 2401.01921; the paper calls LAPACK / cuSOLVER per
// block), by one-sided Jacobi (Hestenes 1958; Demmel and Veselic, SIAM J.
// Matrix Anal. Appl. 13, 1992):
//
//  * each block's shorter dimension gives c working vectors x_p of length r
//    (the columns of M when it has no more columns than rows, else its rows),
//    stored as the rows of X (c x r, row-major), and an accumulator J (c x c)
//    starting at the identity;
//  * a pair (p, q) with alpha = |x_p|^2, beta = |x_q|^2, gamma = x_p . x_q is
//    rotated by the angle that makes it orthogonal: zeta = (beta - alpha) /
//    (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 /
//    sqrt(1 + t^2), s = c t; x_p <- c x_p - s x_q, x_q <- s x_p + c x_q, and
//    the same on the rows p, q of J;
//  * a sweep visits every pair once, in the round-robin ("circle") order:
//    c' - 1 rounds of c'/2 disjoint pairs (c' = c rounded up to even; the
//    pad index pairs with nobody).  One launch per round over the pairs of
//    every block; a pair whose |gamma| is below 1e-15 sqrt(alpha beta) is left
//    as it is; each launch records the largest |gamma| / sqrt(alpha beta) it
//    met, and the host stops after a sweep whose largest value is small
//    (jacobi_coop_kernel runs all rounds and sweeps in one cooperative launch
//    with grid barriers between rounds, when the device allows it);
//  * then sigma_p = |x_p|, and X = J M^T (or J M): the singular vectors are
//    x_p / sigma_p on one side and the rows of J on the other.
// Blocks of 16 or more vectors go through a column-pivoted Householder QR
// first and the sweeps run on the rows of its triangular factor (see the QR
// preconditioning section below); the output has the same form.
// All arithmetic is FP64.  Block reductions use a fixed order (deterministic).
#include "tnx_internal.h"

namespace {

constexpr int JT = 256;   // threads per pair

__device__ __forceinline__ double block_sum3(double& a, double& b, double& c, double* sh) {
  // three sums at once over the CTA, fixed order; results broadcast in a, b, c
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if (lane == 0) {
    sh[wid] = a;
    sh[8 + wid] = b;
    sh[16 + wid] = c;
  }
  __syncthreads();
  a = b = c = 0.0;
  for (int w = 0; w < JT / 32; ++w) {
    a += sh[w];
    b += sh[8 + w];
    c += sh[16 + w];
  }
  __syncthreads();
  return a;
}

__global__ void __launch_bounds__(JT) jacobi_round_kernel(const SvdGroup* __restrict__ groups,
                                                          const int2* __restrict__ slots, int nslots, int round,
                                                          unsigned long long* maxoff) {
  tnx_grid_dependency();
  __shared__ double sh[24];
  __shared__ double s_cs[2];
  __shared__ int s_skip;
  for (int si = blockIdx.x; si < nslots; si += gridDim.x) {
    const int2 sl = slots[si];
    const SvdGroup g = groups[sl.x];
    const int cp = g.c + (g.c & 1);   // c rounded up to even
    if (cp < 2) continue;
    const int kk = round % (cp - 1);
    const int i = sl.y;
    int p, q;
    if (i == 0) {
      p = kk;
      q = cp - 1;
    } else {
      p = (kk + i) % (cp - 1);
      q = (kk - i + cp - 1) % (cp - 1);
    }
    if (p > q) { const int t = p; p = q; q = t; }
    if (q >= g.c) continue;           // the pad index
    double* xp = g.X + (int64_t)p * g.r;
    double* xq = g.X + (int64_t)q * g.r;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int64_t e = threadIdx.x; e < g.r; e += JT) {
      const double u = xp[e], v = xq[e];
      a = fma(u, u, a);
      b = fma(v, v, b);
      c = fma(u, v, c);
    }
    block_sum3(a, b, c, sh);
    if (threadIdx.x == 0) {
      int skip = 1;
      if (a > 0.0 && b > 0.0) {
        const double off = fabs(c) / sqrt(a * b);
        atomicMax(maxoff, (unsigned long long)__double_as_longlong(off));
        if (off > 1e-15) {
          skip = 0;
          const double zeta = (b - a) / (2.0 * c);
          const double az = fabs(zeta);
          double t = az > 1e100 ? 0.5 / az : 1.0 / (az + sqrt(1.0 + az * az));
          if (zeta < 0.0) t = -t;
          const double cs = 1.0 / sqrt(1.0 + t * t);
          s_cs[0] = cs;
          s_cs[1] = cs * t;
        }
      }
      s_skip = skip;
    }
    __syncthreads();
    if (!s_skip) {
      const double cs = s_cs[0], sn = s_cs[1];
      for (int64_t e = threadIdx.x; e < g.r; e += JT) {
        const double u = xp[e], v = xq[e];
        xp[e] = cs * u - sn * v;
        xq[e] = sn * u + cs * v;
      }
      double* jp = g.J + (int64_t)p * g.c;
      double* jq = g.J + (int64_t)q * g.c;
      for (int e = threadIdx.x; e < g.c; e += JT) {
        const double u = jp[e], v = jq[e];
        jp[e] = cs * u - sn * v;
        jq[e] = sn * u + cs * v;
      }
    }
    __syncthreads();   // s_cs / s_skip are rewritten by the next slot
  }
}

// All sweeps of every block in one cooperative launch (all CTAs resident at
// once, which the launch checks): each warp of the grid takes pairs of a
// round across every block (pair i of round k as in jacobi_round_kernel), and
// a grid barrier separates the rounds.  One warp per CTA: the FP64 pipe
// (about two fused multiply-adds per clock per SM on this part) bounds a
// round, so its pairs go to as many SMs as there are pairs.  After each sweep
// the CTAs read the largest squared relative off-diagonal of that sweep
// (offmax[sweep], zeroed by the host) behind a barrier and all stop together
// once it is at most tol2 (the launcher squares tol).  The barrier is one
// 64-bit arrival counter that only grows (a release add to arrive, acquire
// loads to wait); every wait on it is bounded (about a second of clock): on
// expiry the CTA sets *status and leaves, and so do the others at their next
// barrier.  sweeps_out[0] receives the number of sweeps run.
constexpr long long BAR_LIMIT = 2000000000LL;

__device__ bool grid_barrier(unsigned long long* count, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    // every CTA passes the same barriers in the same order, so the count
    // before this arrival lies in [k G, (k+1) G) for barrier k of a grid of
    // G CTAs; the barrier opens when it reaches (k+1) G
    int ok = 1;
    unsigned long long old;
    asm volatile("atom.add.release.gpu.u64 %0, [%1], 1;" : "=l"(old) : "l"(count) : "memory");
    const unsigned long long target = (old / gridDim.x + 1) * (unsigned long long)gridDim.x;
    const long long t0 = clock64();
    for (unsigned it = 1;; ++it) {
      unsigned long long cur;
      asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(cur) : "l"(count) : "memory");
      if (cur >= target) break;
      if ((it & 31u) != 0) continue;   // the error word and the clock every 32 polls
      if (*(volatile int*)status != 0) {
        ok = 0;
        break;
      }
      if (clock64() - t0 > BAR_LIMIT) {
        atomicExch(status, 1);
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
  // butterfly: every lane ends with the same bits (each step adds two partial
  // sums, which commutes exactly)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int CJT = 32;   // threads per CTA of the cooperative kernel: one pair-warp per CTA, so that the
                          // pairs of a round spread over as many SMs (and FP64 pipes) as there are pairs

// One rotation of the pair (p, q) of block g by one warp: the three dots, the
// test and the rotation of jacobi_round_kernel, the test on the squared
// relative off-diagonal (kept in off_w) and the rotation angle from one root.
// VB: vector entries per lane held in registers (8 or 16, vectors of up to 256
// or 512 entries; the launchers take the smaller width that holds the longest
// vector of the launch, and the same for applying Q); longer vectors stream.
template <int VB>
__device__ __forceinline__ void jacobi_pair(const SvdGroup& g, int p, int q, int lane, double& off_w) {
  double* xp = g.X + (int64_t)p * g.r;
  double* xq = g.X + (int64_t)q * g.r;
  double* jp = g.J + (int64_t)p * g.c;
  double* jq = g.J + (int64_t)q * g.c;
  // vectors and J rows of up to 32 VB entries stay in registers between
  // the dots and the rotation: every load of the pair is issued at once
  // (one trip to L2 instead of one per 32 entries)
  const bool in_regs = g.r <= 32 * VB && g.c <= 32 * VB;
  double u[VB], v[VB], ju[VB], jv[VB];
  double a = 0.0, b = 0.0, c = 0.0;
  if (in_regs) {
#pragma unroll
    for (int k = 0; k < VB; ++k) {
      const int e = lane + 32 * k;
      u[k] = e < g.r ? xp[e] : 0.0;
      v[k] = e < g.r ? xq[e] : 0.0;
      ju[k] = e < g.c ? jp[e] : 0.0;
      jv[k] = e < g.c ? jq[e] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < VB; ++k) {
      a = fma(u[k], u[k], a);
      b = fma(v[k], v[k], b);
      c = fma(u[k], v[k], c);
    }
  } else {
#pragma unroll 4
    for (int64_t e = lane; e < g.r; e += 32) {
      const double uu = xp[e], vv = xq[e];
      a = fma(uu, uu, a);
      b = fma(vv, vv, b);
      c = fma(uu, vv, c);
    }
  }
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  if (!(a > 0.0 && b > 0.0)) return;
  // squared relative off-diagonal; the same tests as |gamma| / sqrt(alpha beta)
  // against 1e-15 and tol, with one FP64 division instead of a root and two
  const double ab = a * b, c2 = c * c;
  off_w = fmax(off_w, c2 / ab);
  if (c2 <= 1e-30 * ab) return;
  // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) with zeta = d / (2 gamma), d = beta - alpha,
  // multiplied through by 2 |gamma|: one root, one division and one reciprocal root
  const double d = b - a;
  double t;
  if (fabs(d) < 1e150 && fabs(c) < 1e150) {
    t = 2.0 * c / (d + copysign(sqrt(fma(d, d, 4.0 * c2)), d));
  } else {   // squares out of range: the quotient form
    const double zeta = d / (2.0 * c), az = fabs(zeta);
    t = az > 1e100 ? 0.5 / az : 1.0 / (az + sqrt(1.0 + az * az));
    if (zeta < 0.0) t = -t;
  }
  const double cs = rsqrt(fma(t, t, 1.0)), sn = cs * t;
  if (in_regs) {
#pragma unroll
    for (int k = 0; k < VB; ++k) {
      const int e = lane + 32 * k;
      if (e < g.r) {
        xp[e] = cs * u[k] - sn * v[k];
        xq[e] = sn * u[k] + cs * v[k];
      }
      if (e < g.c) {
        jp[e] = cs * ju[k] - sn * jv[k];
        jq[e] = sn * ju[k] + cs * jv[k];
      }
    }
  } else {
#pragma unroll 4
    for (int64_t e = lane; e < g.r; e += 32) {
      const double uu = xp[e], vv = xq[e];
      xp[e] = cs * uu - sn * vv;
      xq[e] = sn * uu + cs * vv;
    }
#pragma unroll 4
    for (int e = lane; e < g.c; e += 32) {
      const double uu = jp[e], vv = jq[e];
      jp[e] = cs * uu - sn * vv;
      jq[e] = sn * uu + cs * vv;
    }
  }
}

template <int VB>
__global__ void __launch_bounds__(CJT) jacobi_coop_kernel(const SvdGroup* __restrict__ groups,
                                                         const int2* __restrict__ slots, int nslots, int maxcp,
                                                         int max_sweeps, double tol2, unsigned long long* offmax,
                                                         unsigned long long* bar, int* status, int* sweeps_out) {
  // one warp per pair: the pairs of a round run side by side over the whole grid
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (CJT / 32) + (threadIdx.x >> 5), nwarps = gridDim.x * (CJT / 32);
  int sw = 0;
  bool ok = true;
  while (ok && sw < max_sweeps) {
    double off_w = 0.0;   // this warp's largest squared relative off-diagonal of the sweep
    for (int round = 0; round < maxcp - 1 && ok; ++round) {
      for (int si = gw; si < nslots; si += nwarps) {
        const int2 sl = slots[si];
        const SvdGroup g = groups[sl.x];
        const int cp = g.c + (g.c & 1);   // >= 2: a block of one vector has no slot
        const int kk = round % (cp - 1);
        const int i = sl.y;
        int p, q;
        if (i == 0) {
          p = kk;
          q = cp - 1;
        } else {
          p = (kk + i) % (cp - 1);
          q = (kk - i + cp - 1) % (cp - 1);
        }
        if (p > q) { const int t = p; p = q; q = t; }
        if (q < g.c) jacobi_pair<VB>(g, p, q, lane, off_w);   // q = cp - 1 >= c: the pad index
      }
      // one atomic per warp and sweep, before the sweep's last barrier
      if (round == maxcp - 2 && lane == 0 && off_w > 0.0)
        atomicMax(&offmax[sw], (unsigned long long)__double_as_longlong(off_w));
      ok = grid_barrier(bar, status);
    }
    if (!ok) break;
    const double off = __longlong_as_double((long long)*(volatile unsigned long long*)&offmax[sw]);
    ++sw;
    if (off <= tol2) break;   // every warp reads the same value behind the last barrier
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) sweeps_out[0] = sw;
}

// ---------------------------------------------------------------------------
// QR preconditioning (Drmac and Veselic, SIAM J. Matrix Anal. Appl. 29, 2008):
// one-sided Jacobi on the rows of the triangular factor of a column-pivoted
// QR needs far fewer sweeps than on the block itself when the singular values
// are graded (as in a DMRG wavefunction), since those rows are already close
// to orthogonal.  With A = X^T (r x c) and A P = Q R:
//   R = Jr^T Sigma W (Jacobi on the rows of R), so A = (Q Jr^T) Sigma (W P^T):
//   the left singular vectors of A are u_p = Q Jr[p,:]^T, the right ones the
//   rows of W with their columns put back through P.
// The QR is Householder's, in the form of LAPACK's dlarfg: for the pivot
// column x = A[k.., k], beta = -sign(x_0) |x|, tau = (beta - x_0) / beta,
// v = (1, x_1 / (x_0 - beta), ...), H = I - tau v v^T, H x = beta e_0 (tau = 0
// when x_1.. = 0); the pivot is the column with the largest remaining norm.

// Reflector of the column x[0 .. len): all lanes get beta, tau, scale (v_i =
// x_i scale for i >= 1).  The same lanes read the same entries every time, so
// each call on the same data returns the same bits.
__device__ __forceinline__ void reflector(const double* x, int len, int lane, double& beta, double& tau,
                                          double& scale) {
  double s = 0.0;
  for (int i = lane; i < len; i += 32)
    if (i > 0) s = fma(x[i], x[i], s);
  s = warp_sum(s);
  const double x0 = x[0];
  if (s == 0.0) {
    beta = x0;
    tau = 0.0;
    scale = 0.0;
    return;
  }
  const double nrm = sqrt(fma(x0, x0, s));
  beta = x0 >= 0.0 ? -nrm : nrm;
  tau = (beta - x0) / beta;
  scale = 1.0 / (x0 - beta);
}

// Writes the reflector of pivot position k (vector u) in place: X[u][k] =
// beta (the diagonal of R), X[u][k+i] = v_i for i >= 1, tau[k].  Called once
// nothing reads that column any more.
__device__ void reflector_store(const SvdQr& q, int k, int u, int lane) {
  double* x = q.X + (int64_t)u * q.r + k;
  const int len = q.r - k;
  double beta, tau, scale;
  reflector(x, len, lane, beta, tau, scale);
  __syncwarp();   // every lane has read x[0] before lane 0 replaces it
  for (int i = lane; i < len; i += 32) x[i] = i == 0 ? beta : x[i] * scale;
  if (lane == 0) q.tau[k] = tau;
}

// The pivoted QR of every block: a slot is (block, position j); step k runs
// behind a grid barrier.  Every warp of a block reads the same trailing norms
// and picks the same pivot (largest, lowest position on ties), so the
// permutation needs no exchange; positions and norms alternate between two
// buffers from step to step.  The warp of position k records the pivot and
// stores the reflector of step k - 1 (and, at the last step, that of step
// k); the warps of positions j > k apply the step-k reflector to their vector
// and write its new trailing norm, summed from the updated entries.
__global__ void __launch_bounds__(CJT) qr_coop_kernel(const SvdQr* __restrict__ qs, const int2* __restrict__ slots,
                                                      int nslots, int maxc, unsigned long long* bar, int* status) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (CJT / 32) + (threadIdx.x >> 5), nwarps = gridDim.x * (CJT / 32);
  for (int si = gw; si < nslots; si += nwarps) {
    const int2 sl = slots[si];
    const SvdQr q = qs[sl.x];
    const double* x = q.X + (int64_t)sl.y * q.r;
    double s = 0.0;
    for (int i = lane; i < q.r; i += 32) s = fma(x[i], x[i], s);
    s = warp_sum(s);
    if (lane == 0) {
      q.nrm[sl.y] = s;
      q.pos[sl.y] = sl.y;
    }
  }
  bool ok = grid_barrier(bar, status);
  for (int k = 0; k < maxc && ok; ++k) {
    const int cur = k & 1, nxt = cur ^ 1;
    for (int si = gw; si < nslots; si += nwarps) {
      const int2 sl = slots[si];
      const SvdQr q = qs[sl.x];
      const int j = sl.y;
      if (k >= q.c || j < k) continue;
      const double* nr = q.nrm + (int64_t)cur * q.c;
      const int32_t* ps = q.pos + (int64_t)cur * q.c;
      double best = -1.0;
      int bp = q.c;
      for (int i = k + lane; i < q.c; i += 32) {
        const double v = nr[i];
        if (v > best) {
          best = v;
          bp = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        if (ob > best || (ob == best && op < bp)) {
          best = ob;
          bp = op;
        }
      }
      if (bp >= q.c) bp = k;   // no comparable norm (NaN): no exchange
      const int pv = ps[bp], kv = ps[k];
      if (j == k) {
        if (lane == 0) q.perm[k] = pv;
        if (k > 0) reflector_store(q, k - 1, q.perm[k - 1], lane);
        if (k == q.c - 1) reflector_store(q, k, pv, lane);
        continue;
      }
      const int vj = j == bp ? kv : ps[j];
      const double* xp = q.X + (int64_t)pv * q.r + k;
      double* a = q.X + (int64_t)vj * q.r + k;
      const int len = q.r - k;
      double beta, tau, scale;
      reflector(xp, len, lane, beta, tau, scale);
      double ns = 0.0;
      if (tau != 0.0) {
        double w = 0.0;
        for (int i = lane; i < len; i += 32) w = fma(i == 0 ? 1.0 : xp[i] * scale, a[i], w);
        w = warp_sum(w);
        const double tw = tau * w;
        for (int i = lane; i < len; i += 32) {
          const double ai = fma(-tw, i == 0 ? 1.0 : xp[i] * scale, a[i]);
          a[i] = ai;
          if (i > 0) ns = fma(ai, ai, ns);
        }
      } else {
        for (int i = lane; i < len; i += 32)
          if (i > 0) ns = fma(a[i], a[i], ns);
      }
      ns = warp_sum(ns);
      if (lane == 0) {
        q.nrm[(int64_t)nxt * q.c + j] = ns;
        q.pos[(int64_t)nxt * q.c + j] = vj;
      }
    }
    ok = grid_barrier(bar, status);
  }
}

// Xr[p][j] = R[p][j] = X[perm[j]][p] for j >= p (0 below the diagonal), Jr = I
__global__ void qr_gather_r_kernel(const SvdQr* __restrict__ qs, int nq) {
  tnx_grid_dependency();
  for (int gi = blockIdx.y; gi < nq; gi += gridDim.y) {
    const SvdQr q = qs[gi];
    const int64_t n = (int64_t)q.c * q.c;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
      const int p = (int)(e / q.c), j = (int)(e % q.c);
      q.Xr[e] = j >= p ? q.X[(int64_t)q.perm[j] * q.r + p] : 0.0;
      q.Jr[e] = p == j ? 1.0 : 0.0;
    }
  }
}

// One warp per (block, vector p), after the Jacobi on the rows of R:
// sigma_p = |Xr[p,:]|; J[p][perm[i]] = Xr[p][i] / sigma_p (the right singular
// vector of A, 0 when sigma_p = 0); Xf[p,:] = sigma_p Q Jr[p,:]^T, with Q
// applied as H_0 H_1 ... H_{c-1} to (Jr[p,:], 0, ..., 0).  Lane l keeps the
// entries e = l (mod 32) of z throughout, in registers when r <= 32 VB.
template <int VB>
__global__ void qr_apply_kernel(const SvdQr* __restrict__ qs, const int2* __restrict__ vecs, int nvec) {
  tnx_grid_dependency();
  const int lane = threadIdx.x & 31;
  for (int vi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); vi < nvec; vi += gridDim.x * (blockDim.x >> 5)) {
    const int2 gv = vecs[vi];
    const SvdQr q = qs[gv.x];
    const int p = gv.y, c = q.c, r = q.r;
    const double* xr = q.Xr + (int64_t)p * c;
    double s = 0.0;
    for (int i = lane; i < c; i += 32) s = fma(xr[i], xr[i], s);
    s = warp_sum(s);
    const double sg = sqrt(s), inv = sg > 0.0 ? 1.0 / sg : 0.0;
    for (int i = lane; i < c; i += 32) q.J[(int64_t)p * c + q.perm[i]] = xr[i] * inv;
    if (lane == 0) q.sigma[p] = sg;
    const double* jr = q.Jr + (int64_t)p * c;
    double* xf = q.Xf + (int64_t)p * r;
    if (r <= 32 * VB) {
      double z[VB];
#pragma unroll
      for (int m = 0; m < VB; ++m) {
        const int e = lane + 32 * m;
        z[m] = e < c ? jr[e] : 0.0;
      }
      for (int k = c - 1; k >= 0; --k) {
        const double tk = q.tau[k];
        if (tk == 0.0) continue;
        const double* v = q.X + (int64_t)q.perm[k] * r;   // v_e for e > k; v_k = 1
        double vv[VB];
        double w = 0.0;
#pragma unroll
        for (int m = 0; m < VB; ++m) {
          const int e = lane + 32 * m;
          vv[m] = e == k ? 1.0 : (e > k && e < r ? v[e] : 0.0);
          w = fma(vv[m], z[m], w);
        }
        w = warp_sum(w);
        const double tw = tk * w;
#pragma unroll
        for (int m = 0; m < VB; ++m) z[m] = fma(-tw, vv[m], z[m]);
      }
#pragma unroll
      for (int m = 0; m < VB; ++m) {
        const int e = lane + 32 * m;
        if (e < r) xf[e] = sg * z[m];
      }
    } else {
      for (int e = lane; e < r; e += 32) xf[e] = e < c ? jr[e] : 0.0;
      for (int k = c - 1; k >= 0; --k) {
        const double tk = q.tau[k];
        if (tk == 0.0) continue;
        const double* v = q.X + (int64_t)q.perm[k] * r;
        double w = 0.0;
        for (int e = lane; e < r; e += 32)
          if (e >= k) w = fma(e == k ? 1.0 : v[e], xf[e], w);
        w = warp_sum(w);
        const double tw = tk * w;
        for (int e = lane; e < r; e += 32)
          if (e >= k) xf[e] = fma(-tw, e == k ? 1.0 : v[e], xf[e]);
      }
      for (int e = lane; e < r; e += 32) xf[e] *= sg;
    }
  }
}

// J = identity for every group (one CTA per group row block)
__global__ void jacobi_init_kernel(const SvdGroup* __restrict__ groups, int ngroups) {
  tnx_grid_dependency();
  for (int gi = blockIdx.y; gi < ngroups; gi += gridDim.y) {
    const SvdGroup g = groups[gi];
    const int64_t n = (int64_t)g.c * g.c;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
      g.J[e] = (e / g.c == e % g.c) ? 1.0 : 0.0;
  }
}

// sigma_p = |x_p| for every vector of every group: one warp per vector
__global__ void vector_norms_kernel(const SvdGroup* __restrict__ groups, const int2* __restrict__ vecs, int nvec) {
  tnx_grid_dependency();
  const int lane = threadIdx.x & 31;
  for (int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < nvec; v += gridDim.x * (blockDim.x >> 5)) {
    const int2 gv = vecs[v];
    const SvdGroup g = groups[gv.x];
    const double* x = g.X + (int64_t)gv.y * g.r;
    double a = 0.0;
    for (int64_t e = lane; e < g.r; e += 32) a = fma(x[e], x[e], a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) g.sigma[gv.y] = sqrt(a);
  }
}

// Kept singular triplet k of a group: U column k (m rows, ld = kept) and V^T
// row k (n columns); the vector x_p / sigma_p goes to one side and the row p of
// J to the other; scale (sigma or 1) multiplies the U or the V^T side.
__global__ void svd_extract_kernel(const SvdOut* __restrict__ outs, int nout) {
  tnx_grid_dependency();
  for (int oi = blockIdx.x; oi < nout; oi += gridDim.x) {
    const SvdOut o = outs[oi];
    const SvdGroup g = o.g;
    const double sig = g.sigma[o.p];
    const double inv = sig > 0.0 ? 1.0 / sig : 0.0;
    const double* x = g.X + (int64_t)o.p * g.r;
    const double* j = g.J + (int64_t)o.p * g.c;
    // vectors are the columns of M: U gets x / sigma (length r = m), V^T gets j (length c = n);
    // vectors are the rows of M:    U gets j (length c = m),         V^T gets x / sigma (length r = n)
    const double su = o.absorb == 2 ? sig : 1.0;
    const double sv = o.absorb == 1 ? sig : 1.0;
    if (o.cols_are_vectors) {
      for (int64_t e = threadIdx.x; e < g.r; e += blockDim.x) o.U[e * o.ldu + o.k] = x[e] * inv * su;
      for (int64_t e = threadIdx.x; e < g.c; e += blockDim.x) o.Vt[(int64_t)o.k * o.ldv + e] = j[e] * sv;
    } else {
      for (int64_t e = threadIdx.x; e < g.c; e += blockDim.x) o.U[e * o.ldu + o.k] = j[e] * su;
      for (int64_t e = threadIdx.x; e < g.r; e += blockDim.x) o.Vt[(int64_t)o.k * o.ldv + e] = x[e] * inv * sv;
    }
    if (threadIdx.x == 0 && o.S) o.S[(int64_t)o.k * o.lds + o.k] = sig;
  }
}

// 2-D block copies: dst[i * dld + j] = src[i * sld + j] (or, transposed,
// dst[j * dld + i] = src[i * sld + j]) for i < rows, j < cols
__global__ void copy2d_kernel(const Copy2D* __restrict__ tasks, int ntasks) {
  tnx_grid_dependency();
  for (int ti = blockIdx.x; ti < ntasks; ti += gridDim.x) {
    const Copy2D t = tasks[ti];
    const int64_t n = (int64_t)t.rows * t.cols;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
      const int64_t i = e / t.cols, j = e % t.cols;
      const double v = t.src[i * t.sld + j];
      if (t.trans) t.dst[j * t.dld + i] = v;
      else t.dst[i * t.dld + j] = v;
    }
  }
}

}  // namespace

cudaError_t tnx_launch_jacobi_init(const SvdGroup* groups, int ngroups, cudaStream_t st) {
  if (ngroups <= 0) return cudaSuccess;
  const cudaError_t le = tnx_launch(jacobi_init_kernel, dim3(64, ngroups < 65535 ? ngroups : 65535), dim3(256), 0, st,
                                    groups, ngroups);
  if (le != cudaSuccess) return le;
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_jacobi_round(const SvdGroup* groups, const int2* slots, int nslots, int round,
                                    unsigned long long* maxoff, cudaStream_t st) {
  if (nslots <= 0) return cudaSuccess;
  const int grid = nslots < 152 * 8 ? nslots : 152 * 8;
  const cudaError_t le = tnx_launch(jacobi_round_kernel, dim3(grid), dim3(JT), 0, st, groups, slots, nslots, round,
                                    maxoff);
  if (le != cudaSuccess) return le;
  tnx_note_launch(1);
  return cudaGetLastError();
}

namespace {
template <int VB>
cudaError_t launch_jacobi_coop(const SvdGroup* groups, const int2* slots, int nslots, int maxcp, int max_sweeps,
                               double tol, unsigned long long* offmax, unsigned long long* bar, int* status,
                               int* sweeps_out, cudaStream_t st) {
  int dev = 0, nsm = 0, per_sm = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_coop_kernel<VB>, CJT, 0);
  if (e != cudaSuccess) return e;
  if (!coop || per_sm < 1) return cudaErrorNotSupported;
  int grid = nsm * (per_sm < 4 ? per_sm : 4);
  const int need = (nslots + CJT / 32 - 1) / (CJT / 32);   // one warp per pair of a round
  if (grid > need) grid = need;
  double tol2 = tol * tol;   // the kernel compares squared relative off-diagonals
  void* args[] = {(void*)&groups, (void*)&slots, (void*)&nslots, (void*)&maxcp, (void*)&max_sweeps, (void*)&tol2,
                  (void*)&offmax, (void*)&bar, (void*)&status, (void*)&sweeps_out};
  e = cudaLaunchCooperativeKernel((const void*)jacobi_coop_kernel<VB>, dim3(grid), dim3(CJT), args, 0, st);
  if (e != cudaSuccess) return e;
  tnx_note_launch(1);
  return cudaSuccess;
}
}  // namespace

cudaError_t tnx_launch_jacobi_coop(const SvdGroup* groups, const int2* slots, int nslots, int maxcp, int maxlen,
                                   int max_sweeps, double tol, unsigned long long* offmax, unsigned long long* bar,
                                   int* status, int* sweeps_out, cudaStream_t st) {
  if (nslots <= 0 || maxcp < 2) return cudaSuccess;
  return maxlen <= 32 * 8 ? launch_jacobi_coop<8>(groups, slots, nslots, maxcp, max_sweeps, tol, offmax, bar, status,
                                                  sweeps_out, st)
                          : launch_jacobi_coop<16>(groups, slots, nslots, maxcp, max_sweeps, tol, offmax, bar, status,
                                                   sweeps_out, st);
}

cudaError_t tnx_launch_qr_coop(const SvdQr* qs, const int2* slots, int nslots, int maxc, unsigned long long* bar,
                               int* status, cudaStream_t st) {
  if (nslots <= 0 || maxc < 1) return cudaSuccess;
  int dev = 0, nsm = 0, per_sm = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_coop_kernel, CJT, 0);
  if (e != cudaSuccess) return e;
  if (!coop || per_sm < 1) return cudaErrorNotSupported;
  int grid = nsm * (per_sm < 4 ? per_sm : 4);
  if (grid > nslots) grid = nslots;   // one warp per slot of a step
  void* args[] = {(void*)&qs, (void*)&slots, (void*)&nslots, (void*)&maxc, (void*)&bar, (void*)&status};
  e = cudaLaunchCooperativeKernel((const void*)qr_coop_kernel, dim3(grid), dim3(CJT), args, 0, st);
  if (e != cudaSuccess) return e;
  tnx_note_launch(1);
  return cudaSuccess;
}

cudaError_t tnx_launch_qr_gather_r(const SvdQr* qs, int nq, int maxc, cudaStream_t st) {
  if (nq <= 0) return cudaSuccess;
  int bx = (int)(((int64_t)maxc * maxc + 255) / 256);
  if (bx > 64) bx = 64;
  if (bx < 1) bx = 1;
  const cudaError_t le = tnx_launch(qr_gather_r_kernel, dim3(bx, nq < 65535 ? nq : 65535), dim3(256), 0, st, qs, nq);
  if (le != cudaSuccess) return le;
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_qr_apply(const SvdQr* qs, const int2* vecs, int nvec, int maxr, cudaStream_t st) {
  if (nvec <= 0) return cudaSuccess;
  // one warp per vector, two warps per CTA: the vectors spread over the SMs' FP64 pipes
  const int grid = (nvec + 1) / 2;
  const cudaError_t le = maxr <= 32 * 8 ? tnx_launch(qr_apply_kernel<8>, dim3(grid), dim3(64), 0, st, qs, vecs, nvec)
                                        : tnx_launch(qr_apply_kernel<16>, dim3(grid), dim3(64), 0, st, qs, vecs, nvec);
  if (le != cudaSuccess) return le;
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_vector_norms(const SvdGroup* groups, const int2* vecs, int nvec, cudaStream_t st) {
  if (nvec <= 0) return cudaSuccess;
  const int grid = (nvec + 7) / 8 < 152 * 8 ? (nvec + 7) / 8 : 152 * 8;
  const cudaError_t le = tnx_launch(vector_norms_kernel, dim3(grid), dim3(256), 0, st, groups, vecs, nvec);
  if (le != cudaSuccess) return le;
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_svd_extract(const SvdOut* outs, int nout, cudaStream_t st) {
  if (nout <= 0) return cudaSuccess;
  const int grid = nout < 152 * 8 ? nout : 152 * 8;
  const cudaError_t le = tnx_launch(svd_extract_kernel, dim3(grid), dim3(128), 0, st, outs, nout);
  if (le != cudaSuccess) return le;
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_copy2d(const Copy2D* tasks, int ntasks, cudaStream_t st) {
  if (ntasks <= 0) return cudaSuccess;
  const int grid = ntasks < 152 * 8 ? ntasks : 152 * 8;
  const cudaError_t le = tnx_launch(copy2d_kernel, dim3(grid), dim3(256), 0, st, tasks, ntasks);
  if (le != cudaSuccess) return le;
  tnx_note_launch(1);
  return cudaGetLastError();
}
