// Fused charge-sector matching kernel (integer, exact).
//
// For one pairwise contraction of block-sparse tensors (Sec. 7 of
// arXiv 2401.01921: sum over common labels, only zero-flux blocks stored;
// grouping of equal charges as in the bond combine of Sec. 6.2.2) it builds
// the tables that turn the contraction into one dense product per total
// charge g of the contracted legs:
//   - a K tuple (sector indices of the contracted legs, A's leg order) is valid
//     if some block of A and some block of B carry it; its group is the flux
//     of those legs seen from A; groups ascend lexicographically by charge;
//   - rows (free-A tuples of A blocks with a valid K tuple), valid K tuples
//     and columns (free-B tuples) are ordered lexicographically inside their
//     group; offsets are prefix sums of the products of degeneracies;
//   - amap[block of A] = (group, row offset, K offset), bmap likewise, -1 if unused.
//
// Tuple spaces are enumerated in mixed radix (first leg most significant), so
// increasing tuple id is lexicographic order.  One CTA of 1024 threads runs
// all phases, separated by __syncthreads(); the weighted prefix sums per group
// use a stable per-thread-chunk counting scan.  Runs once per plan.
#include "tnx_internal.h"

namespace {

constexpr int T = 1024;

__device__ int64_t tuple_dim(const MatchArgs& a, const MatchLeg* legs, int nl, int64_t id) {
  int64_t d = 1;
  for (int l = nl - 1; l >= 0; --l) {
    int s = (int)(id % legs[l].nsec);
    id /= legs[l].nsec;
    d *= a.deg[legs[l].sec_base + s];
  }
  return d;
}

__device__ int64_t tuple_id(const int32_t* q, const int32_t* pos, const MatchLeg* legs, int nl) {
  int64_t id = 0;
  for (int l = 0; l < nl; ++l) id = id * legs[l].nsec + q[pos[l]];
  return id;
}

__device__ bool sectors_in_range(const int32_t* q, const int32_t* pos, const MatchLeg* legs, int nl) {
  for (int l = 0; l < nl; ++l) {
    const int32_t v = q[pos[l]];
    if (v < 0 || v >= legs[l].nsec) return false;
  }
  return true;
}

// charge index of K tuple `id` in the dense charge space (component 0 most significant)
__device__ int64_t kcharge_index(const MatchArgs& a, int64_t id) {
  int32_t g[TNX_MAXSYM];
  for (int c = 0; c < a.nsym; ++c) g[c] = 0;
  for (int l = a.nk - 1; l >= 0; --l) {
    int s = (int)(id % a.kleg[l].nsec);
    id /= a.kleg[l].nsec;
    const int32_t* q = a.kcharge + (int64_t)(a.kleg[l].sec_base + s) * a.nsym;
    for (int c = 0; c < a.nsym; ++c) g[c] += q[c];
  }
  int64_t cs = 0;
  for (int c = 0; c < a.nsym; ++c) {
    int v = g[c];
    if (a.zn[c] > 0) v = ((v % a.zn[c]) + a.zn[c]) % a.zn[c];
    if (v < a.clo[c] || v >= a.clo[c] + a.crange[c]) return -1;   // host bounds violated
    cs = cs * a.crange[c] + (v - a.clo[c]);
  }
  return cs;
}

// Stable weighted prefix sum per group over items [0, n) in index order.
// grp(i) < 0: item skipped.  off[i] = sum of weights of earlier items of the
// same group; totals[g] = group total.  tmp: T * G int64 scratch.
template <class GrpF, class WF>
__device__ void group_scan(int64_t n, int G, GrpF grp, WF weight, int64_t* off, int64_t* totals, int64_t* tmp) {
  const int t = threadIdx.x;
  const int64_t c0 = n * t / T, c1 = n * (t + 1) / T;
  for (int g = 0; g < G; ++g) tmp[(int64_t)t * G + g] = 0;
  for (int64_t i = c0; i < c1; ++i) {
    int g = grp(i);
    if (g >= 0) tmp[(int64_t)t * G + g] += weight(i);
  }
  __syncthreads();
  for (int g = t; g < G; g += T) {
    int64_t run = 0;
    for (int c = 0; c < T; ++c) {
      int64_t v = tmp[(int64_t)c * G + g];
      tmp[(int64_t)c * G + g] = run;
      run += v;
    }
    totals[g] = run;
  }
  __syncthreads();
  for (int64_t i = c0; i < c1; ++i) {
    int g = grp(i);
    if (g >= 0) {
      off[i] = tmp[(int64_t)t * G + g];
      tmp[(int64_t)t * G + g] += weight(i);
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(T) match_kernel(MatchArgs a) {
  const int t = threadIdx.x;
  __shared__ int32_t s_G;
  __shared__ int32_t s_bad;
  __shared__ int32_t s_scan[T];
  if (t == 0) s_bad = 0;

  // phase 0: clear
  for (int64_t i = t; i < a.kspace; i += T) { a.kpres[i] = 0; a.kgroup[i] = -1; }
  for (int64_t i = t; i < a.faspace; i += T) a.rgroup[i] = -1;
  for (int64_t i = t; i < a.fbspace; i += T) a.cgroup[i] = -1;
  for (int64_t i = t; i < a.cspace; i += T) a.cspres[i] = 0;
  __syncthreads();

  // phase 1: which K tuples occur in A and in B.  Every sector index of a
  // block is checked against its leg first: an index out of range would
  // address outside the tuple-space arrays, so such a block is skipped and
  // the call reports status 3 without writing any table.
  for (int64_t b = t; b < a.nA; b += T) {
    const int32_t* q = a.qA + b * a.rA;
    if (!sectors_in_range(q, a.kposA, a.kleg, a.nk) || !sectors_in_range(q, a.fposA, a.faleg, a.nfa)) {
      s_bad = 1;
      continue;
    }
    atomicOr(&a.kpres[tuple_id(q, a.kposA, a.kleg, a.nk)], 1);
  }
  for (int64_t b = t; b < a.nB; b += T) {
    const int32_t* q = a.qB + b * a.rB;
    if (!sectors_in_range(q, a.kposB, a.kleg, a.nk) || !sectors_in_range(q, a.fposB, a.fbleg, a.nfb)) {
      s_bad = 1;
      continue;
    }
    atomicOr(&a.kpres[tuple_id(q, a.kposB, a.kleg, a.nk)], 2);
  }
  __syncthreads();
  if (s_bad) {
    if (t == 0) { *a.status = 3; *a.ngroups = 0; }
    return;
  }

  // phase 2: mark the charges of valid K tuples
  for (int64_t k = t; k < a.kspace; k += T)
    if (a.kpres[k] == 3) {
      int64_t cs = kcharge_index(a, k);
      if (cs >= 0) a.cspres[cs] = 1;
      else *a.status = 2;
    }
  __syncthreads();

  // phase 3: exclusive scan of the charge-presence array -> group ids (ascending charge)
  {
    int64_t chunk = (a.cspace + T - 1) / T;
    int64_t c0 = chunk * t, c1 = min(a.cspace, c0 + chunk);
    int32_t local = 0;
    for (int64_t i = c0; i < c1; ++i) local += a.cspres[i];
    s_scan[t] = local;
    __syncthreads();
    if (t == 0) {
      int32_t run = 0;
      for (int i = 0; i < T; ++i) { int32_t v = s_scan[i]; s_scan[i] = run; run += v; }
      s_G = run;
    }
    __syncthreads();
    int32_t run = s_scan[t];
    for (int64_t i = c0; i < c1; ++i) {
      a.csgid[i] = a.cspres[i] ? run : -1;
      run += a.cspres[i];
    }
  }
  __syncthreads();
  const int G = s_G;
  if (G > a.gmax) {
    if (t == 0) { *a.status = 1; *a.ngroups = G; }
    return;
  }

  // phase 4: group of each valid K tuple; charges of each group
  for (int64_t k = t; k < a.kspace; k += T)
    if (a.kpres[k] == 3) {
      int64_t cs = kcharge_index(a, k);
      if (cs >= 0) a.kgroup[k] = a.csgid[cs];
    }
  for (int64_t i = t; i < a.cspace; i += T) {
    int g = a.csgid[i];
    if (g >= 0) {
      int64_t r = i;
      for (int c = a.nsym - 1; c >= 0; --c) {
        a.charges[(int64_t)g * a.nsym + c] = (int32_t)(r % a.crange[c]) + a.clo[c];
        r /= a.crange[c];
      }
    }
  }
  __syncthreads();

  // phase 5: K offsets inside each group
  int64_t* totK = a.scan_tmp + (int64_t)T * a.gmax;            // gmax entries after the T*gmax block
  group_scan(a.kspace, G, [&](int64_t i) { return a.kgroup[i]; },
             [&](int64_t i) { return tuple_dim(a, a.kleg, a.nk, i); }, a.koff, totK, a.scan_tmp);

  // phase 6: rows and columns inherit the group of their block's valid K tuple
  for (int64_t b = t; b < a.nA; b += T) {
    const int32_t* q = a.qA + b * a.rA;
    int g = a.kgroup[tuple_id(q, a.kposA, a.kleg, a.nk)];
    if (g >= 0) a.rgroup[tuple_id(q, a.fposA, a.faleg, a.nfa)] = g;
  }
  for (int64_t b = t; b < a.nB; b += T) {
    const int32_t* q = a.qB + b * a.rB;
    int g = a.kgroup[tuple_id(q, a.kposB, a.kleg, a.nk)];
    if (g >= 0) a.cgroup[tuple_id(q, a.fposB, a.fbleg, a.nfb)] = g;
  }
  __syncthreads();
  int64_t* totM = totK + a.gmax;
  int64_t* totN = totM + a.gmax;
  group_scan(a.faspace, G, [&](int64_t i) { return a.rgroup[i]; },
             [&](int64_t i) { return tuple_dim(a, a.faleg, a.nfa, i); }, a.roff, totM, a.scan_tmp);
  group_scan(a.fbspace, G, [&](int64_t i) { return a.cgroup[i]; },
             [&](int64_t i) { return tuple_dim(a, a.fbleg, a.nfb, i); }, a.coff, totN, a.scan_tmp);

  // phase 7: per-block maps and group sizes
  for (int64_t b = t; b < a.nA; b += T) {
    const int32_t* q = a.qA + b * a.rA;
    int64_t k = tuple_id(q, a.kposA, a.kleg, a.nk);
    int g = a.kgroup[k];
    int64_t* o = a.amap + 3 * b;
    if (g >= 0) { o[0] = g; o[1] = a.roff[tuple_id(q, a.fposA, a.faleg, a.nfa)]; o[2] = a.koff[k]; }
    else { o[0] = -1; o[1] = -1; o[2] = -1; }
  }
  for (int64_t b = t; b < a.nB; b += T) {
    const int32_t* q = a.qB + b * a.rB;
    int64_t k = tuple_id(q, a.kposB, a.kleg, a.nk);
    int g = a.kgroup[k];
    int64_t* o = a.bmap + 3 * b;
    if (g >= 0) { o[0] = g; o[1] = a.koff[k]; o[2] = a.coff[tuple_id(q, a.fposB, a.fbleg, a.nfb)]; }
    else { o[0] = -1; o[1] = -1; o[2] = -1; }
  }
  for (int g = t; g < G; g += T) {
    a.mkn[3 * g + 0] = totM[g];
    a.mkn[3 * g + 1] = totK[g];
    a.mkn[3 * g + 2] = totN[g];
  }
  if (t == 0) { *a.ngroups = G; }
}

}  // namespace

cudaError_t tnx_launch_match(const MatchArgs& a, cudaStream_t st) {
  match_kernel<<<1, T, 0, st>>>(a);
  tnx_note_launch(1);
  return cudaGetLastError();
}
