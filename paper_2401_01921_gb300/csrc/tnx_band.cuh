// Device helpers for band tiles (see tnx_internal.h): blocks that share the
// rows of a row-major matrix on one side, staged a tile of rows at a time in
// shared memory.  Used by the relayout kernel and by the fused skinny product.
#pragma once

#include "tnx_internal.h"

namespace tnx_band {

// n / d for 0 <= n < 2^22 and d >= 1, with inv = 1.0f / d: the float estimate
// is off by at most one, which the remainder test corrects.
__device__ __forceinline__ int qdiv(int n, int d, float inv) {
  int q = __float2int_rz((float)n * inv);
  const int r = n - q * d;
  if (r < 0) --q;
  else if (r >= d) ++q;
  return q;
}

// One band member, as seen from the current tile (kept in shared memory).
struct Member {
  long long nbase;      // narrow-side offset of the member's element (p0, q0, 0)
  int nslot, wcol;      // narrow-side slot; first column in the rows
  int t0, t1;           // tile extents of the two fastest dimensions (narrow order)
  int s0, s1, s2;       // narrow-side strides, fastest dimension first
  int w0, w1, w2;       // shared-memory strides, same order
  float inv0, inv1;
  int nelem3;           // tile extent of the slowest dimension
};

// Member m (legs P, Q, I) for the tile p in [p0, p0 + tP), q in [q0, q0 + tQ):
// its narrow side is the source when `gather`, else the destination; (wP, wQ)
// are the shared-memory strides of P and Q (I has stride 1, from column wcol).
// The dimensions are walked in the order of the narrow-side strides, so that
// consecutive threads touch consecutive narrow-side addresses.
__device__ inline Member stage(const CopyTask& m, bool gather, int p0, int q0, int tP, int tQ, int wP, int wQ) {
  const int32_t* ns = gather ? m.sstride : m.dstride;
  int ext[3] = {tP, tQ, m.shape[2]}, nst[3] = {ns[0], ns[1], ns[2]}, sst[3] = {wP, wQ, 1};
  int ord[3] = {0, 1, 2};
  auto key = [&](int d) { return ext[d] > 1 ? (long long)nst[d] : (1ll << 40) + d; };
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2 - a; ++b)
      if (key(ord[b]) > key(ord[b + 1])) {
        const int x = ord[b];
        ord[b] = ord[b + 1];
        ord[b + 1] = x;
      }
  Member b;
  b.nslot = gather ? m.src_slot : m.dst_slot;
  b.nbase = (gather ? m.src_off : m.dst_off) + (long long)p0 * nst[0] + (long long)q0 * nst[1];
  b.wcol = m.wcol;
  b.t0 = ext[ord[0]];
  b.t1 = ext[ord[1]];
  b.nelem3 = ext[ord[2]];
  b.s0 = nst[ord[0]];
  b.s1 = nst[ord[1]];
  b.s2 = nst[ord[2]];
  b.w0 = sst[ord[0]];
  b.w1 = sst[ord[1]];
  b.w2 = sst[ord[2]];
  b.inv0 = 1.0f / (float)b.t0;
  b.inv1 = 1.0f / (float)b.t1;
  return b;
}

// pre[k] = elements of members 0..k-1 in this tile, pre[nt] = all (computed by
// warp `warp`; the caller synchronises before and after).
__device__ inline void prefix(const Member* mem, int nt, int* pre, int warp = 0) {
  if ((int)(threadIdx.x >> 5) != warp) return;
  const int lane = threadIdx.x & 31;
  int run = 0;
  for (int k0 = 0; k0 < nt; k0 += 32) {
    const int k = k0 + lane;
    int x = k < nt ? mem[k].t0 * mem[k].t1 * mem[k].nelem3 : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (k < nt) pre[k + 1] = run + x;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) pre[0] = 0;
}

constexpr int kUnroll = 4;   // elements per thread with their loads in flight together

// Every member element of the tile between its narrow side and shared memory:
// GATHER: buf[s] = narrow[n] (a negative slot reads zeros); else narrow[n] = buf[s].
// U elements per thread are addressed and loaded before any is stored.
template <int NT, bool GATHER, int U = kUnroll>
__device__ inline void move(const Member* mem, const int* pre, int nt, double* buf, double* const* __restrict__ slots) {
  const int total = pre[nt];
  for (int ebase = threadIdx.x; ebase < total; ebase += NT * U) {
    double v[U];
    int so[U];
    double* dp[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = ebase + u * NT;
      so[u] = -1;
      if (e < total) {
        int lo = 0, hi = nt;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (pre[mid] <= e) lo = mid; else hi = mid;
        }
        const Member& m = mem[lo];
        const int l = e - pre[lo];
        const int e12 = qdiv(l, m.t0, m.inv0), e0 = l - e12 * m.t0;
        const int e2 = qdiv(e12, m.t1, m.inv1), e1 = e12 - e2 * m.t1;
        const int no = e0 * m.s0 + e1 * m.s1 + e2 * m.s2;
        so[u] = e0 * m.w0 + e1 * m.w1 + e2 * m.w2 + m.wcol;
        if (GATHER) {
          v[u] = m.nslot >= 0 ? __ldg(slots[m.nslot] + m.nbase + no) : 0.0;
        } else {
          dp[u] = slots[m.nslot] + m.nbase + no;
          v[u] = buf[so[u]];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (so[u] < 0) continue;
      if (GATHER) buf[so[u]] = v[u];
      else *dp[u] = v[u];
    }
  }
}

}  // namespace tnx_band
