// Split-precision grouped GEMM on the tcgen05 tensor cores (sm_103a).
//
// The fused-sector products of a pairwise contraction (Sec. 7 of
// arXiv 2401.01921; the paper runs them as FP64 library GEMMs) are computed to
// FP64 accuracy from 16-bit tensor-core products with the error-free slicing
// of Ozaki, Ogita, Oishi and Rump (Numer. Algorithms 59, 2012):
//
//  * every row of A (and every column of B) gets a common power-of-two scale
//    2^(E+1) from the exponent E of its largest entry; an entry x becomes the
//    signed fixed-point integer v = round(x 2^(F-E-2)), |v| <= 2^(F-1),
//    F = n*beta, written in n balanced base-2^beta digits
//    v = sum_i d_i 2^(beta(n-1-i)), d_i in [-2^(beta-1), 2^(beta-1)]; each
//    digit is an integer, exact in BF16 or FP16;
//  * the product sum_k a_k b_k becomes sum over digit pairs (i, j); pairs with
//    the same level t = i + j share one FP32 accumulator in tensor memory; all
//    pairs with t <= n-1 are formed (terms below 2^-(beta n) are dropped); the
//    accumulators of consecutive levels sit in consecutive TMEM columns, so
//    one MMA of A slice i against the stacked B slices 0..n-1-i feeds all of
//    its levels at once;
//  * the K loop runs in chunks of KC = 640: with beta = 7 a level sums at
//    most n * KC * 64^2 < 2^24, so every FP32 accumulation is exact; after
//    each chunk the levels are read out of tensor memory and added, exactly,
//    into a 64-bit integer fixed-point accumulator
//    I = sum_t L_t 2^(beta(n-1-t));
//  * the result is rounded once: C = I * 2^(E_r + E_c + 2 - 2(F-1) + beta(n-1)).
// The only error is the rounding of each operand to F-1 bits below its
// row / column maximum and the dropped levels: about 2^-40 relative to
// max|row| * max|col| * K.
//
// Kernel layout: 128 x 64 output tiles, 10 warps per CTA: warp 0 issues the
// bulk copies (the TMA engine, cp.async.bulk) of pre-tiled slices into a
// 3-stage shared-memory ring, warp 1 issues tcgen05.mma (one elected lane),
// warps 2-9 (two per quarter of the TMEM lanes, each taking half of the
// tile's columns) drain tensor memory (tcgen05.ld) into the integer accumulators
// and write FP64.  Operands sit in global memory already in the canonical
// no-swizzle K-major core-matrix layout, so a stage is one contiguous copy.
// Every wait on an mbarrier is bounded (about a second of clock); a wait that
// runs out records an error code and the CTA winds down without hanging.
//
// The same kernel, instantiated with TF = true, is the one-pass TF32 variant:
// one "slice" per operand holding the entry scaled by its row (column) power of
// two and rounded to TF32 (10 explicit mantissa bits, nearest-even), 16 K
// values (64 bytes) per stage and row, tcgen05.mma.kind::tf32 with FP32
// accumulation per 640-long K chunk, chunks summed in FP64 by the epilogue.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tnx_internal.h"

namespace {

constexpr int TM = 128;            // tile rows (A)
constexpr int TK = 32;             // K per stage
constexpr int KC = 640;            // K per exact chunk
constexpr int STAGES = 3;
constexpr int MAXN = 6;            // slices
constexpr int ATILE = TM * TK * 2; // bytes of one A slice tile (8 KB)
// tile columns (B rows): TNV = 64 (wide) or 32 (narrow); one B slice tile is TNV * TK * 2 bytes
constexpr long long WAIT_LIMIT = 2000000000LL;   // clock cycles (~1 s)
constexpr int EPI_WARPS = 8;       // epilogue warps: two per TMEM lane quarter, each takes half the columns
constexpr int SPLIT_THREADS = 32 * (2 + EPI_WARPS);

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// bounded wait; returns false (and records `code`) if the limit runs out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, int32_t* status, int code,
                                          volatile int* abort_flag) {
  const long long t0 = clock64();
  while (!mbar_try(bar, phase)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_LIMIT) {
      atomicExch(status, code);
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: no swizzle, K-major, core matrices of
// 8 rows x 16 bytes; LBO = stride between core matrices along K (128 B),
// SBO = stride between 8-row groups (512 B for a 32-wide K tile).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
  return d;                 // base offset 0, swizzle none
}

// instruction descriptor, kind::f16: D f32, A/B bf16 (1) or f16 (0), both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t instr_desc(int f16, int n) {
  const uint32_t ab = f16 ? 0u : 1u;
  return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// (value of a 64-bit integer) * 2^e rounded to nearest-even FP64, with integer
// operations only (the FP64 pipe of this part is slow); results below the
// normal range flush to zero.
__device__ __forceinline__ double i64_scaled_to_double(long long v, int e) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
  unsigned long long u = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll(u);
  u <<= lz;                                   // leading one at bit 63
  unsigned long long mant = u >> 11;          // 53 bits
  const unsigned long long rem = u & 0x7FFull;
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) mant += 1;
  int ex = 63 - lz + e;
  if (mant >> 53) {
    mant >>= 1;
    ex += 1;
  }
  const int biased = ex + 1023;
  if (biased <= 0) return __longlong_as_double((long long)sign);
  if (biased >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
  return __longlong_as_double((long long)(sign | ((unsigned long long)biased << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// The same value through the hardware conversion: __ll2double_rn rounds v to
// 53 bits (nearest-even) and adding e to the exponent field is the exact
// scaling by 2^e while the result stays normal; outside that range the
// integer routine above decides.
__device__ __forceinline__ double i64_scaled_fast(long long v, int e) {
  if (v == 0) return 0.0;
  const long long bits = __double_as_longlong(__ll2double_rn(v));
  const int ex = (int)((bits >> 52) & 0x7FF) + e;
  if (ex >= 1 && ex <= 2046) return __longlong_as_double(bits + ((long long)e << 52));
  return i64_scaled_to_double(v, e);
}

// kind::tf32: D f32, A/B tf32 (format 2), both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t instr_desc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------ slicing
// 64 * (1 + 128 + ... + 128^5): added to a signed 42-bit value it makes every
// base-128 digit non-negative (digit i of the sum is digit i of v plus 64)
constexpr long long DIGIT_BIAS = 64LL * ((1LL << 42) - 1) / 127;

// Slices of the packed operands, one CTA (8 warps) per work item.  Rows are
// taken in groups of 8 (rows past an operand's end give zero slices); in a
// warp, lane = (row in group) * 4 + (8-column group).  A job gives each group
// SliceJob::wpg warps (1, 2, 4 or 8: more for longer rows), so an item is
// 8 / wpg groups.  For a group, first the biased exponent of each row's
// largest |x| (lanes of a row scan every 4 * wpg-th entry's exponent field,
// then the lanes and the group's warps combine), stored for the GEMM epilogue;
// then the group's 32-wide K tiles are sliced, the warps of the group taking
// every wpg-th tile, 8 entries per lane, 16 bytes per slice per lane written
// in the tiled core-matrix layout the GEMM copies in.
// With KX (K balancing), entry k counts as x * 2^(kx_sign * E_k), E_k the
// exponent of column k's largest entry in A: A's columns are scaled by 2^-E_k
// and B's rows by 2^E_k, exactly, so the product is unchanged while a row of
// A (column of B) whose entries scale differently along K keeps its bits.
// Only exponents move: the digits of x * 2^s are those of x with the
// effective exponent E + s.
__device__ __forceinline__ int kx_shift(int raw, int sign) {
  return raw > 0 ? sign * (raw - 1023) : 0;   // raw: biased exponent, 0 for a zero column
}

// With VEC (vector mode, no K balancing) a row's entries come from the
// Lanczos vector through the row table, scaled by *inv, and the scaled values
// are written out as the next basis vector (VecSrc).
template <bool F16, bool KX, bool VEC>
__global__ void __launch_bounds__(256) slice_rows_kernel(const SliceJob* __restrict__ jobs,
                                                         const int2* __restrict__ items, int64_t total,
                                                         double* const* __restrict__ slots, VecSrc vs) {
  static_assert(!(KX && VEC), "vector mode slices without K balancing");
  tnx_grid_dependency();
  if constexpr (VEC) {
    if (*(volatile const int32_t*)(vs.state + 1) != 0) return;   // the solve has stopped
  }
  const double vinv = VEC ? *vs.inv : 1.0;
  __shared__ int s_max[8][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int r8 = lane >> 2, kq = lane & 3;
  constexpr int F = MAXN * 7;   // six digits of 7 bits (checked by the launcher)
  for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
    const int2 item = items[w];   // (job, first 8-row group)
    const SliceJob& j = jobs[item.x];
    const int wpg = j.wpg;                        // uniform over the CTA
    const int sub = wid / wpg, wl = wid - sub * wpg;
    const int64_t ngroups = ((int64_t)j.rows + j.tile_rows - 1) / j.tile_rows * (j.tile_rows / 8);
    const int64_t rg = (int64_t)item.y + sub;
    const int KT = (j.K + TK - 1) / TK;
    const int64_t row = rg * 8 + r8;
    const bool live = rg < ngroups && row < j.rows;
    int64_t voff = 0;   // vector mode: offset of the row's K entries in the vector
    const double* src;
    if constexpr (VEC) {
      voff = live ? vs.rowtab[j.src_off + row] : 0;
      src = vs.w + voff;
    } else {
      src = slots[j.src_slot] + j.src_off + row * j.ld;
    }
    // row exponent: the largest (effective) exponent field; eight independent
    // loads of the high words in flight per lane
    const uint32_t* src_hi = (const uint32_t*)src + 1;
    const int32_t* kxp = KX ? (const int32_t*)slots[j.kx_slot] + j.kx_off : nullptr;
    const int kstart = wl * 4 + kq, kstep = 4 * wpg;
    constexpr int ZROW = KX ? -(1 << 20) : 0;   // no nonzero entry
    int mx = ZROW;
    if (live)
      for (int k0 = kstart; k0 < j.K; k0 += 8 * kstep) {
        uint32_t h[8];
        int sx[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int k = k0 + u * kstep;
          if constexpr (VEC)
            h[u] = k < j.K ? (uint32_t)((unsigned long long)__double_as_longlong(src[k] * vinv) >> 32) : 0u;
          else
            h[u] = k < j.K ? src_hi[2 * k] : 0u;
          if constexpr (KX) sx[u] = k < j.K ? kxp[k] : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int eb = (int)((h[u] >> 20) & 0x7FFu);
          if constexpr (KX) {
            if (eb != 0) mx = max(mx, eb + kx_shift(sx[u], j.kx_sign));
          } else {
            mx = max(mx, eb);
          }
        }
      }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (wpg > 1) {
      if (kq == 0) s_max[wid][r8] = mx;
      __syncthreads();
      for (int q = sub * wpg; q < sub * wpg + wpg; ++q) mx = max(mx, s_max[q][r8]);
      __syncthreads();   // s_max is rewritten by the next item
    }
    if (rg >= ngroups) continue;   // a group past the job's last one
    const int eb_r = mx;
    const bool nonzero_row = eb_r != ZROW;
    if (live && kq == 0 && wl == 0) ((int32_t*)slots[j.exp_slot])[j.exp_off + row] = nonzero_row ? eb_r : 0;
    const int tile_rows = j.tile_rows;
    const int64_t mt = row / tile_rows;
    const int rin = (int)(row % tile_rows);
    const int64_t tile_bytes = (int64_t)tile_rows * TK * 2;
    char* base = (char*)slots[j.dst_slot] + j.dst_off_bytes;
    const int64_t inner = (int64_t)(rin >> 3) * 512 + kq * 128 + (rin & 7) * 16;
    // Digits of one K tile (8 entries per lane); the loads of the lane's next
    // tile are issued before the current one is converted.
    // With KX the K-balancing words of the tile come along (each group's region
    // is padded to whole K tiles and 16-byte aligned).
    const int kt0 = wl, kts = wpg;
    unsigned long long cur[8];
    int4 ckx[2];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kt0 * TK + kq * 8 + e;
      if constexpr (VEC) {
        cur[e] = 0ull;
        if (live && kt0 < KT && k < j.K) {
          const double x = src[k] * vinv;
          vs.vdst[voff + k] = x;
          cur[e] = (unsigned long long)__double_as_longlong(x);
        }
      } else {
        cur[e] = (live && kt0 < KT && k < j.K) ? (unsigned long long)__double_as_longlong(src[k]) : 0ull;
      }
    }
    if constexpr (KX) {
      const bool ok = live && kt0 < KT;
      ckx[0] = ok ? *(const int4*)(kxp + kt0 * TK + kq * 8) : make_int4(0, 0, 0, 0);
      ckx[1] = ok ? *(const int4*)(kxp + kt0 * TK + kq * 8 + 4) : make_int4(0, 0, 0, 0);
    }
    for (int kt = kt0; kt < KT; kt += kts) {
      unsigned long long nxt[8];
      int4 nkx[2];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = (kt + kts) * TK + kq * 8 + e;
        if constexpr (VEC) {
          nxt[e] = 0ull;
          if (live && kt + kts < KT && k < j.K) {
            const double x = src[k] * vinv;
            vs.vdst[voff + k] = x;
            nxt[e] = (unsigned long long)__double_as_longlong(x);
          }
        } else {
          nxt[e] = (live && kt + kts < KT && k < j.K) ? (unsigned long long)__double_as_longlong(src[k]) : 0ull;
        }
      }
      if constexpr (KX) {
        const bool ok = live && kt + kts < KT;
        nkx[0] = ok ? *(const int4*)(kxp + (kt + kts) * TK + kq * 8) : make_int4(0, 0, 0, 0);
        nkx[1] = ok ? *(const int4*)(kxp + (kt + kts) * TK + kq * 8 + 4) : make_int4(0, 0, 0, 0);
      }
      int sh[8];
      if constexpr (KX) {
        const int raw[8] = {ckx[0].x, ckx[0].y, ckx[0].z, ckx[0].w, ckx[1].x, ckx[1].y, ckx[1].z, ckx[1].w};
#pragma unroll
        for (int e = 0; e < 8; ++e) sh[e] = kx_shift(raw[e], j.kx_sign);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) sh[e] = 0;
      }
      uint32_t sl[MAXN][4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        float f[2][MAXN];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const unsigned long long bits = cur[e + h];
          const int eb = (int)((bits >> 52) & 0x7FF);
          // |x| 2^(F-E-2) rounded half up: m53 * 2^-rs with rs = 54 - F + E_r - E >= 12
          unsigned long long fix = 0;
          if (eb != 0 && nonzero_row) {
            const unsigned long long m53 = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
            const int rs = 54 - F + (eb_r - (eb + sh[e + h]));
            fix = rs >= 64 ? 0ull : ((m53 >> (rs - 1)) + 1ull) >> 1;
          }
          // Balanced base-128 digits of the signed value v (|v| <= 2^41): with
          // u = v + 64 * sum_i 128^i >= 0, the plain 7-bit digits e_i of u give
          // d_i = e_i - 64 in [-64, 63] (the top digit takes the rest, at most 64),
          // and sum_i d_i 128^i = v.
          const long long v = (bits >> 63) ? -(long long)fix : (long long)fix;
          const unsigned long long u = (unsigned long long)(v + DIGIT_BIAS);
          const uint32_t lo = (uint32_t)(u & 0x1FFFFFull), hi = (uint32_t)(u >> 21);
          uint32_t dg[MAXN];   // e_i of slice i (slice 0 = most significant)
          dg[5] = lo & 127u;
          dg[4] = (lo >> 7) & 127u;
          dg[3] = lo >> 14;
          dg[2] = hi & 127u;
          dg[1] = (hi >> 7) & 127u;
          dg[0] = hi >> 14;
          // d = e - 64 exactly as FP32: in the binade of 1.5 * 2^23 one unit of the
          // bit pattern is one unit of value, so (bits 0x4B400000 + d) - 1.5 * 2^23 = d
#pragma unroll
          for (int i = 0; i < MAXN; ++i) f[h][i] = __int_as_float(0x4B3FFFC0 + (int)dg[i]) - 12582912.0f;
        }
#pragma unroll
        for (int i = 0; i < MAXN; ++i) {
          // |d| <= 64 is exact in BF16 (the top half of the FP32 word) and in FP16
          if constexpr (F16) {
            const __half2 hh = __floats2half2_rn(f[0][i], f[1][i]);
            sl[i][e >> 1] = *(const uint32_t*)&hh;
          } else {
            sl[i][e >> 1] = __byte_perm(__float_as_uint(f[0][i]), __float_as_uint(f[1][i]), 0x7632);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < MAXN; ++i) {
        uint4 v = make_uint4(sl[i][0], sl[i][1], sl[i][2], sl[i][3]);
        *(uint4*)(base + ((mt * KT + kt) * MAXN + i) * tile_bytes + inner) = v;
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) cur[e] = nxt[e];
      if constexpr (KX) {
        ckx[0] = nkx[0];
        ckx[1] = nkx[1];
      }
    }
  }
}

// Zeroes the K-balancing words of every job (whole K tiles), one CTA per job.
__global__ void kexp_zero_kernel(const KexpJob* __restrict__ jobs, int njobs, double* const* __restrict__ slots) {
  tnx_grid_dependency();
  for (int q = blockIdx.x; q < njobs; q += gridDim.x) {
    const KexpJob& j = jobs[q];
    int32_t* kx = (int32_t*)slots[j.kx_slot] + j.kx_off;
    const int n = (j.K + TK - 1) / TK * TK;
    for (int i = threadIdx.x; i < n; i += blockDim.x) kx[i] = 0;
  }
}

// Column maxima of the exponent fields of A: an item is 32 K indices (one per
// lane) by 64 rows (eight per warp, loads in flight together); the warps
// combine in shared memory and one atomicMax per K index leaves the CTA.
__global__ void __launch_bounds__(256) kexp_kernel(const KexpJob* __restrict__ jobs, const int4* __restrict__ items,
                                                   int64_t nitems, double* const* __restrict__ slots) {
  tnx_grid_dependency();
  __shared__ int s_mx[8][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int4 it = items[w];   // (job, first K index, first row, -)
    const KexpJob& j = jobs[it.x];
    const int k = it.y + lane;
    int mx = 0;
    if (k < j.K) {
      const uint32_t* hi = (const uint32_t*)(slots[j.src_slot] + j.src_off) + 1;
      uint32_t h[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int r = it.z + wid + 8 * u;
        h[u] = r < j.rows ? hi[2 * ((int64_t)r * j.ld + k)] : 0u;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) mx = max(mx, (int)((h[u] >> 20) & 0x7FFu));
    }
    s_mx[wid][lane] = mx;
    __syncthreads();
    if (wid == 0) {
#pragma unroll
      for (int q = 1; q < 8; ++q) mx = max(mx, s_mx[q][lane]);
      if (k < j.K && mx > 0) atomicMax((int32_t*)slots[j.kx_slot] + j.kx_off + k, mx);
    }
    __syncthreads();
  }
}

// TF32 operands of the one-pass variant: one CTA (8 warps) per item of eight
// 8-row groups, one group per warp; lane = (row in group) * 4 + (4-column
// group).  A row is scaled by 2^-E (E: unbiased exponent of its largest |x|,
// stored for the epilogue like the split path's), rounded to 11 significant
// bits (nearest-even) straight from the FP64 bits, and written as FP32 words
// in the tiled core-matrix layout, 16 K values (64 bytes) per tile row.
// Entries more than 2^126 below their row maximum flush to zero.
__device__ __forceinline__ uint32_t tf32_word(unsigned long long bits, int eb_r) {
  const int eb = (int)((bits >> 52) & 0x7FF);
  const uint32_t sign = (uint32_t)(bits >> 63) << 31;
  if (eb == 0 || eb_r == 0) return sign;
  int ef = eb - eb_r + 127;
  unsigned long long keep = ((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> 42;   // 11 bits
  const unsigned long long rem = bits & ((1ull << 42) - 1), half = 1ull << 41;
  if (rem > half || (rem == half && (keep & 1ull))) keep += 1;
  if (keep >> 11) {
    keep >>= 1;
    ef += 1;
  }
  if (ef <= 0) return sign;
  return sign | ((uint32_t)ef << 23) | ((uint32_t)(keep & 0x3FFull) << 13);
}

__global__ void __launch_bounds__(256) tf32_rows_kernel(const SliceJob* __restrict__ jobs,
                                                        const int2* __restrict__ items, int64_t total,
                                                        double* const* __restrict__ slots) {
  tnx_grid_dependency();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int r8 = lane >> 2, kq = lane & 3;
  constexpr int TKF = 16;   // K values per tile row
  for (int64_t w = blockIdx.x; w < total; w += gridDim.x) {
    const int2 item = items[w];   // (job, first 8-row group)
    const SliceJob& j = jobs[item.x];
    const int64_t ngroups = ((int64_t)j.rows + j.tile_rows - 1) / j.tile_rows * (j.tile_rows / 8);
    const int64_t rg = (int64_t)item.y + wid;
    if (rg >= ngroups) continue;   // uniform over the warp
    const int64_t row = rg * 8 + r8;
    const bool live = row < j.rows;
    const double* src = slots[j.src_slot] + j.src_off + row * j.ld;
    unsigned long long mx = 0;
    if (live)
      for (int k = kq; k < j.K; k += 4) {
        const unsigned long long b = __double_as_longlong(src[k]) & 0x7FFFFFFFFFFFFFFFull;
        mx = b > mx ? b : mx;
      }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = v > mx ? v : mx;
    }
    const int eb_r = (int)(mx >> 52);
    if (live && kq == 0) ((int32_t*)slots[j.exp_slot])[j.exp_off + row] = eb_r;
    const int KT = (j.K + TKF - 1) / TKF;
    const int tile_rows = j.tile_rows;
    const int64_t mt = row / tile_rows;
    const int rin = (int)(row % tile_rows);
    const int64_t tile_bytes = (int64_t)tile_rows * TKF * 4;
    char* base = (char*)slots[j.dst_slot] + j.dst_off_bytes;
    const int64_t inner = (int64_t)(rin >> 3) * 512 + kq * 128 + (rin & 7) * 16;
    for (int kt = 0; kt < KT; ++kt) {
      uint32_t o[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = kt * TKF + kq * 4 + e;
        const unsigned long long bits = (live && k < j.K) ? (unsigned long long)__double_as_longlong(src[k]) : 0ull;
        o[e] = tf32_word(bits, eb_r);
      }
      *(uint4*)(base + (mt * KT + kt) * tile_bytes + inner) = make_uint4(o[0], o[1], o[2], o[3]);
    }
  }
}

// --------------------------------------------------------- split GEMM
struct SplitShared {
  uint64_t full[STAGES], empty[STAGES];
  uint64_t accfull, accempty, done;
  uint32_t tmem_base;
  int abort_flag;
};

// Persistent over tiles: CTA b takes tiles b, b + gridDim.x, ... of the list
// (the host orders it longest-K first, or lays out a per-CTA schedule whose
// holes carry group -1).  Tensor memory and the barriers are set
// up once per CTA; the stage ring and the chunk hand-off between the MMA warp
// and the epilogue warps continue across tiles, so the producer streams the
// next tile's slices while the epilogue drains the current one.
template <int NS, int TNV, bool TF, int MODE>
__global__ void __launch_bounds__(SPLIT_THREADS, 1) split_gemm_kernel(const SplitGroup* __restrict__ groups,
                                                             const GemmTile* __restrict__ tiles, int ntiles, int beta,
                                                             int f16, double* const* __restrict__ slots,
                                                             int32_t* status) {
  tnx_grid_dependency();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* ring = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int BTILE = TNV * TK * 2;
  constexpr int ECOLS = TNV / 2;     // tile columns per epilogue warp
  constexpr int STAGE_BYTES = NS * (ATILE + BTILE);
  SplitShared* sh = (SplitShared*)(ring + STAGES * STAGE_BYTES);
  double (*sh_stage)[4] = (double (*)[4])(ring + STAGES * STAGE_BYTES + ((sizeof(SplitShared) + 15) & ~(size_t)15));
  int* sh_ebc = (int*)(sh_stage + EPI_WARPS * 32);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int TKE = TF ? 16 : TK;   // K values per stage (64 bytes per row either way)
  constexpr int KTPC = KC / TKE;      // K tiles per chunk
  static_assert(!TF || NS == 1, "the TF32 variant has one operand slice");

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&sh->full[s], 1);
      mbar_init(&sh->empty[s], 1);
    }
    mbar_init(&sh->accfull, 1);
    mbar_init(&sh->accempty, EPI_WARPS);
    mbar_init(&sh->done, 1);
    sh->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&sh->tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh->tmem_base;
  volatile int* abort_flag = &sh->abort_flag;

  if (warp == 0) {
    // ---------------- producer: bulk copies of pre-tiled slices
    if (lane == 0) {
      int g = 0;   // global K-tile counter of this CTA
      for (int ti = blockIdx.x; ti < ntiles && !*abort_flag; ti += gridDim.x) {
        const GemmTile tl = tiles[ti];
        if (tl.group < 0) continue;   // a hole of the per-CTA schedule
        const SplitGroup gr = groups[tl.group];
        const int KT = (gr.K + TKE - 1) / TKE;
        const char* Ab = (const char*)slots[gr.a_slot] + gr.a_off_bytes + ((int64_t)(tl.m0 / TM) * KT) * NS * ATILE;
        const char* Bb = (const char*)slots[gr.b_slot] + gr.b_off_bytes + ((int64_t)(tl.n0 / TNV) * KT) * NS * BTILE;
        for (int kt = 0; kt < KT; ++kt, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
          if (g >= STAGES && !mbar_wait(&sh->empty[s], ph ^ 1u, status, 11, abort_flag)) break;
          unsigned char* sa = ring + s * STAGE_BYTES;
          mbar_expect_tx(&sh->full[s], NS * (ATILE + BTILE));
          bulk_g2s(sa, Ab + (int64_t)kt * NS * ATILE, NS * ATILE, &sh->full[s]);
          bulk_g2s(sa + NS * ATILE, Bb + (int64_t)kt * NS * BTILE, NS * BTILE, &sh->full[s]);
        }
      }
      // never leave copies in flight: wait (bounded) for the last issued stages to land
      for (int q = (g > STAGES ? g - STAGES : 0); q < g; ++q) {
        const long long t0 = clock64();
        while (!mbar_try(&sh->full[q % STAGES], (uint32_t)(q / STAGES) & 1u) && clock64() - t0 < WAIT_LIMIT) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int g = 0, chunk = 0;
      bool ok = true;
      for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
        const int tg = tiles[ti].group;
        if (tg < 0) continue;
        const SplitGroup gr = groups[tg];
        const int KT = (gr.K + TKE - 1) / TKE;
        for (int kt = 0; kt < KT; ++kt, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
          const bool first_in_chunk = (kt % KTPC) == 0;
          const bool last_in_chunk = ((kt + 1) % KTPC) == 0 || kt == KT - 1;
          if (first_in_chunk && chunk > 0 && !mbar_wait(&sh->accempty, (uint32_t)(chunk - 1) & 1u, status, 12, abort_flag)) {
            ok = false;
            break;
          }
          if (!mbar_wait(&sh->full[s], ph, status, 13, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(ring + s * STAGE_BYTES);
          const uint32_t sb = sa + NS * ATILE;
          // A slice i meets the B slices j = 0 .. NS-1-i stacked along N (they are
          // consecutive TNV-row tiles, so the stack is one taller K-major operand);
          // its output columns are the accumulators of levels i .. NS-1, also
          // consecutive: one MMA (N <= 256, else two) per A slice and K step.
          // A K step is 32 bytes of every row: 16 values of BF16/FP16, 8 of TF32.
#pragma unroll
          for (int ks = 0; ks < TK / 16; ++ks) {
#pragma unroll
            for (int i = 0; i < NS; ++i) {
              const uint64_t ad = smem_desc(sa + i * ATILE + ks * 256);
              const uint32_t acc = (first_in_chunk && ks == 0 && i == 0) ? 0u : 1u;
              const int nj = NS - i;
              constexpr int PER_MMA = 256 / TNV;   // B slices per MMA (N <= 256)
#pragma unroll
              for (int j0 = 0; j0 < nj; j0 += PER_MMA) {
                const int cnt = (nj - j0) < PER_MMA ? (nj - j0) : PER_MMA;
                const uint64_t bd = smem_desc(sb + j0 * BTILE + ks * 256);
                if constexpr (TF) mma_tf32(tmem + (uint32_t)((i + j0) * TNV), ad, bd, instr_desc_tf32(cnt * TNV), acc);
                else mma_f16(tmem + (uint32_t)((i + j0) * TNV), ad, bd, instr_desc(f16, cnt * TNV), acc);
              }
            }
          }
          mma_commit(&sh->empty[s]);
          if (last_in_chunk) {
            mma_commit(&sh->accfull);
            ++chunk;
          }
        }
      }
      // all MMAs issued by this thread have completed before tensor memory is freed
      mma_commit(&sh->done);
      const long long t0 = clock64();
      while (!mbar_try(&sh->done, 0) && clock64() - t0 < WAIT_LIMIT) {
      }
    }
  } else {
    // ---------------- epilogue: warps 2..9; warp w reads TMEM lanes 32*(w%4) ..
    // (rows of the tile) and one half of the tile's columns
    const int sub = warp & 3;
    const int cb = ((warp - 2) >> 2) * ECOLS;
    int chunk = 0;
    bool ok = true;
    for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
      const GemmTile tl = tiles[ti];
      if (tl.group < 0) continue;
      const SplitGroup gr = groups[tl.group];
      const int KT = (gr.K + TKE - 1) / TKE;
      const int nchunks = (KT + KTPC - 1) / KTPC;
      const int row = tl.m0 + sub * 32 + lane;
      // Row and column exponents are fetched before the first accumulator
      // wait, so their global-load latency hides behind the MMAs.
      double (*stg)[4] = sh_stage + (warp - 2) * 32;
      int* ebc_s = sh_ebc + (warp - 2) * ECOLS;
      const int eb_r = row < gr.M ? ((const int32_t*)slots[gr.ea_slot])[gr.ea_off + row] : 0;
      {
        const int32_t* eb_c = (const int32_t*)slots[gr.eb_slot] + gr.eb_off;
        const int col = tl.n0 + cb + lane;
        if (lane < ECOLS) ebc_s[lane] = col < gr.N ? eb_c[col] : 0;
      }
      long long acc[ECOLS];
      double accd[ECOLS];   // TF32: FP64 sum of the FP32 chunk sums
#pragma unroll
      for (int c = 0; c < ECOLS; ++c) {
        acc[c] = 0;
        accd[c] = 0.0;
      }
      for (int ch = 0; ch < nchunks; ++ch, ++chunk) {
        if (!mbar_wait(&sh->accfull, (uint32_t)chunk & 1u, status, 14, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // all levels of 8 columns in flight at once, one wait per column group
#pragma unroll
        for (int cg = 0; cg < ECOLS / 8; ++cg) {
          uint32_t v[NS][8];
#pragma unroll
          for (int t = 0; t < NS; ++t)
            tmem_ld8(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(t * TNV + cb + cg * 8), v[t]);
          tmem_wait_ld();
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            if constexpr (TF) {
              accd[cg * 8 + c] += (double)__uint_as_float(v[0][c]);
            } else if constexpr (MODE == 2) {
              // MODE 2: every tile of the launch has K <= 160, so each level sum is
              // below 6 * 160 * 64^2 < 2^22, where the FP32 -> int conversion is an
              // exact add of 1.5 * 2^23 on the full-rate ALU, and adjacent levels
              // combine in 32-bit integers before the 64-bit sum
              int d[NS];
#pragma unroll
              for (int t = 0; t < NS; ++t) d[t] = __float_as_int(__uint_as_float(v[t][c]) + 12582912.0f) - 0x4B400000;
              const int lo = d[5] + d[4] * 128, mid = d[3] + d[2] * 128, hi = d[1] + d[0] * 128;   // |.| < 2^30
              acc[cg * 8 + c] += ((long long)hi << 28) + ((long long)mid << 14) + (long long)lo;
            } else {
              long long x = 0;
#pragma unroll
              for (int t = 0; t < NS; ++t)
                x += (long long)__float2int_rn(__uint_as_float(v[t][c])) * (1LL << (beta * (NS - 1 - t)));
              acc[cg * 8 + c] += x;
            }
          }
        }
        tc_fence_before();
        if (lane == 0) mbar_arrive(&sh->accempty);
      }
      if (ok) {
        // Convert and write through a per-warp staging block of 32 rows x 4
        // columns, so each store instruction covers whole 32-byte sectors of
        // eight rows of C instead of one 8-byte word in each of 32 rows.
        // Column c of row r sits at position c ^ ((r >> 2) & 3), which keeps
        // the row-wise writes and the column-wise reads free of bank conflicts.
        __syncwarp();
        double* cbase = slots[gr.c_slot] + gr.c_off;
        // a folded output relayout: column descriptors, destination = the network's output
        // (MODE 1, the folded output relayout: an instantiation of its own, so the
        // plain store path keeps its registers)
        const FinalCol* fcol = MODE == 1 ? (const FinalCol*)slots[gr.fc_slot] + gr.fc_off : nullptr;
        double* obase = MODE == 1 ? slots[gr.out_slot] : nullptr;
        const int r0 = tl.m0 + sub * 32;
#pragma unroll
        for (int c4 = 0; c4 < ECOLS / 4; ++c4) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if constexpr (TF) {
              // operands were scaled by 2^-(E_r) and 2^-(E_c)
              stg[lane][c ^ ((lane >> 2) & 3)] = ldexp(accd[c4 * 4 + c], eb_r + ebc_s[c4 * 4 + c] - 2046);
            } else {
              const int e = eb_r + ebc_s[c4 * 4 + c] - 2044 - 2 * (NS * beta - 1) + beta * (NS - 1);
              stg[lane][c ^ ((lane >> 2) & 3)] = i64_scaled_fast(acc[c4 * 4 + c], e);
            }
          }
          __syncwarp();
          const int cc = lane & 3, col = tl.n0 + cb + c4 * 4 + cc;
          if constexpr (MODE == 1) {
            const FinalCol d = col < gr.N ? fcol[col] : FinalCol{-1, 0};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int rr = q * 8 + (lane >> 2), r = r0 + rr;
              if (r < gr.M && d.off >= 0) obase[d.off + (int64_t)r * d.stride] = stg[rr][cc ^ ((rr >> 2) & 3)];
            }
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int rr = q * 8 + (lane >> 2), r = r0 + rr;
              if (r < gr.M && col < gr.N) cbase[(int64_t)r * gr.ldc + col] = stg[rr][cc ^ ((rr >> 2) & 3)];
            }
          }
          __syncwarp();
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

}  // namespace

cudaError_t tnx_launch_slices(const SliceJob* jobs, const int2* items, int64_t total_items, int nslice, int beta,
                              int f16, double* const* slots, cudaStream_t st, int use_kx) {
  if (total_items <= 0) return cudaSuccess;
  if (nslice != MAXN || beta != 7) return cudaErrorInvalidValue;   // the digit code is specialised
  int64_t blocks = total_items;
  if (blocks > 152 * 8) blocks = 152 * 8;
  {
    const dim3 g((int)blocks), b(256);
    const VecSrc none{nullptr, nullptr, nullptr, nullptr, nullptr};
    const cudaError_t le =
        f16 ? (use_kx ? tnx_launch(slice_rows_kernel<true, true, false>, g, b, 0, st, jobs, items, total_items, slots,
                                   none)
                      : tnx_launch(slice_rows_kernel<true, false, false>, g, b, 0, st, jobs, items, total_items,
                                   slots, none))
            : (use_kx ? tnx_launch(slice_rows_kernel<false, true, false>, g, b, 0, st, jobs, items, total_items,
                                   slots, none)
                      : tnx_launch(slice_rows_kernel<false, false, false>, g, b, 0, st, jobs, items, total_items,
                                   slots, none));
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_slices_vec(const SliceJob* jobs, const int2* items, int64_t total_items, int nslice, int beta,
                                  int f16, double* const* slots, const VecSrc& vs, cudaStream_t st) {
  if (total_items <= 0) return cudaSuccess;
  if (nslice != MAXN || beta != 7) return cudaErrorInvalidValue;   // the digit code is specialised
  if (!vs.rowtab || !vs.w || !vs.vdst || !vs.inv || !vs.state) return cudaErrorInvalidValue;
  int64_t blocks = total_items;
  if (blocks > 152 * 8) blocks = 152 * 8;
  {
    const dim3 g((int)blocks), b(256);
    const cudaError_t le =
        f16 ? tnx_launch(slice_rows_kernel<true, false, true>, g, b, 0, st, jobs, items, total_items, slots, vs)
            : tnx_launch(slice_rows_kernel<false, false, true>, g, b, 0, st, jobs, items, total_items, slots, vs);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_kexp(const KexpJob* jobs, int njobs, const int4* items, int64_t nitems, double* const* slots,
                            cudaStream_t st) {
  if (njobs <= 0 || nitems <= 0) return cudaSuccess;
  cudaError_t le = tnx_launch(kexp_zero_kernel, dim3(njobs < 1024 ? njobs : 1024), dim3(256), 0, st, jobs, njobs,
                              slots);
  if (le != cudaSuccess) return le;
  const int64_t blocks = nitems < 152 * 8 ? nitems : 152 * 8;
  le = tnx_launch(kexp_kernel, dim3((int)blocks), dim3(256), 0, st, jobs, items, nitems, slots);
  if (le != cudaSuccess) return le;
  tnx_note_launch(2);
  return cudaGetLastError();
}

size_t tnx_split_smem_bytes(int nslice, int tn) {
  // alignment slack + stage ring + barriers + epilogue staging (32 rows x 4 doubles
  // per epilogue warp) + column exponents (tn / 2 per epilogue warp)
  return 1024 + (size_t)STAGES * nslice * (ATILE + (size_t)tn * TK * 2) + ((sizeof(SplitShared) + 15) & ~(size_t)15) +
         EPI_WARPS * 32 * 4 * sizeof(double) + EPI_WARPS * (tn / 2) * sizeof(int) + 64;
}

namespace {
template <int TNV, bool TF, int MODE>
cudaError_t launch_split_t(const SplitGroup* groups, const GemmTile* tiles, int ntiles, int beta, int f16,
                           double* const* slots, int32_t* status, cudaStream_t st, int grid) {
  constexpr int NS = TF ? 1 : MAXN;
  const size_t smem = tnx_split_smem_bytes(NS, TNV);
  static int attr_dev = -1;   // the opt-in is per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (attr_dev != dev) {
    e = cudaFuncSetAttribute(split_gemm_kernel<NS, TNV, TF, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  return tnx_launch(split_gemm_kernel<NS, TNV, TF, MODE>, dim3(grid), dim3(SPLIT_THREADS), smem, st,
                    groups, tiles, ntiles, beta, f16, slots, status);
}

// mode: 0 plain stores, 1 folded output relayout, 2 plain stores with the
// short-K level combine (split BF16/FP16 only)
template <int TNV, bool TF>
cudaError_t launch_split(const SplitGroup* groups, const GemmTile* tiles, int ntiles, int beta, int f16,
                         double* const* slots, int32_t* status, cudaStream_t st, int grid, int mode) {
  if (mode == 1) return launch_split_t<TNV, TF, 1>(groups, tiles, ntiles, beta, f16, slots, status, st, grid);
  if constexpr (!TF) {
    if (mode == 2) return launch_split_t<TNV, TF, 2>(groups, tiles, ntiles, beta, f16, slots, status, st, grid);
  }
  return launch_split_t<TNV, TF, 0>(groups, tiles, ntiles, beta, f16, slots, status, st, grid);
}
}  // namespace

cudaError_t tnx_launch_gemm_split(const SplitGroup* groups, const GemmTile* tiles, int ntiles, int nslice, int beta,
                                  int f16, double* const* slots, int32_t* status, cudaStream_t st, int grid, int tn,
                                  int mode) {
  if (ntiles <= 0) return cudaSuccess;
  if (grid <= 0 || grid > ntiles) grid = ntiles;
  if (nslice != MAXN || beta != 7 || (tn != 32 && tn != 64)) return cudaErrorInvalidValue;
  const cudaError_t le =
      tn == 32 ? launch_split<32, false>(groups, tiles, ntiles, beta, f16, slots, status, st, grid, mode)
               : launch_split<64, false>(groups, tiles, ntiles, beta, f16, slots, status, st, grid, mode);
  if (le != cudaSuccess) return le;
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_tf32_rows(const SliceJob* jobs, const int2* items, int64_t total_items, double* const* slots,
                                 cudaStream_t st) {
  if (total_items <= 0) return cudaSuccess;
  int64_t blocks = total_items;
  if (blocks > 152 * 8) blocks = 152 * 8;
  const cudaError_t le = tnx_launch(tf32_rows_kernel, dim3((int)blocks), dim3(256), 0, st, jobs, items, total_items,
                                    slots);
  if (le != cudaSuccess) return le;
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_gemm_tf32(const SplitGroup* groups, const GemmTile* tiles, int ntiles, double* const* slots,
                                 int32_t* status, cudaStream_t st, int grid, int tn, int fold) {
  if (ntiles <= 0) return cudaSuccess;
  if (grid <= 0 || grid > ntiles) grid = ntiles;
  if (tn != 32 && tn != 64) return cudaErrorInvalidValue;
  const cudaError_t le = tn == 32 ? launch_split<32, true>(groups, tiles, ntiles, 0, 0, slots, status, st, grid, fold)
                                  : launch_split<64, true>(groups, tiles, ntiles, 0, 0, slots, status, st, grid, fold);
  if (le != cudaSuccess) return le;
  tnx_note_launch(1);
  return cudaGetLastError();
}
