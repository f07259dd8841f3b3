// Permute-to-GEMM relayout kernel.
//
// The paper's permute is lazy (metadata only) and data moves when a
// contiguous copy is requested (Appendix A, "permute" / "contiguous"), which
// the library does right before each block GEMM (Sec. 7).  Here every block
// of an operand is moved, permuted, straight into its place inside the fused
// operand matrix of its charge group (or, after the last contraction, into
// the canonical block layout of the output tensor).
//
// A task copies one block: per leg a shape, a source stride and a destination
// stride (elements); the legs are ordered so that the last one is contiguous
// in the destination.  The planner cuts large tasks into chunks of at most
// CHUNK elements and packs runs of small tasks (up to PACK of them, CHUNK
// elements in all) into one chunk; one CTA takes one chunk,
// its threads walk destination order so stores coalesce, and loads coalesce
// whenever the source is contiguous along the same leg.  When the source is
// contiguous along another leg, the task is moved in 32 x 32 tiles staged
// through shared memory instead, so both sides coalesce.  Blocks that share
// the rows of a narrow matrix on one side (a packed GEMM operand of K <= 96
// columns they are written into, or a GEMM output of <= 96 columns they are
// read from) move as one band: a tile of whole rows is staged in shared
// memory, the wide side is accessed row by row and each block's other side
// along its own contiguous leg.  Index arithmetic is 32-bit inside a task, and
// an index is split over the legs with multiply-high divisions by the leg
// extents (constants the planner precomputes) instead of hardware integer
// divisions.
#include <algorithm>

#include "tnx_band.cuh"

namespace {

constexpr int CT = 256;

// floor(n / shape[l]) for 0 <= n < 2^31 from the task's precomputed constants
__device__ __forceinline__ int fdiv(int n, uint32_t magic, uint32_t shift) {
  return magic ? (int)(__umulhi((uint32_t)n, magic) >> shift) : n;
}

// Transposing task: the source is contiguous along leg S = t.tleg, the
// destination along the last leg.  View the block as a matrix with one column
// per index of S and one row per index of the other legs (in task order), and
// move it in 32 x 32 tiles through shared memory: loads run along S, stores
// along the rows (consecutive rows are consecutive in the destination).
template <bool SCALED>
__device__ void copy_transpose(const CopyTask& t, int tile, double* const* __restrict__ slots, double (*sm)[33],
                               const double* src_base, double scale, double* vdst_base) {
  const int r = t.rank, S = t.tleg;
  const int ncols = t.shape[S];
  const int nrows = (int)(t.nelem / ncols);
  const int nct = (ncols + 31) >> 5;
  const int r0 = (tile / nct) << 5, c0 = (tile % nct) << 5;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double* src = SCALED ? src_base + t.src_off : (t.src_slot >= 0 ? slots[t.src_slot] + t.src_off : nullptr);
  double* dst = slots[t.dst_slot] + t.dst_off;
  // row index -> (source offset, destination offset) over the legs other than S
  auto bases = [&](int row, int& so, int& dof) {
    so = 0;
    dof = 0;
    for (int l = r - 1; l >= 0; --l) {
      if (l == S) continue;
      const int q = fdiv(row, t.magic[l], t.shift[l]);
      const int rem = row - q * t.shape[l];
      row = q;
      so += rem * t.sstride[l];
      dof += rem * t.dstride[l];
    }
  };
  const int c = c0 + lane;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rr = wid + 8 * i, row = r0 + rr;
    if (row < nrows && c < ncols) {
      int so, dof;
      bases(row, so, dof);
      const double x = src ? __ldg(src + so + c * t.sstride[S]) : 0.0;
      if (SCALED) {
        const double y = x * scale;
        sm[rr][lane] = y;
        if (vdst_base) vdst_base[t.src_off + so + c * t.sstride[S]] = y;
      } else {
        sm[rr][lane] = x;
      }
    }
  }
  __syncthreads();
  const int row = r0 + lane;
  if (row < nrows) {
    int so, dof;
    bases(row, so, dof);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int cc = wid + 8 * i, col = c0 + cc;
      if (col < ncols) dst[dof + col * t.dstride[S]] = sm[lane][cc];
    }
  }
}

// One tile of a band (see tnx_internal.h): rows (p, q) of the wide side for
// p in [p0, p0 + tP), q in [q0, q0 + tQ), all W columns.  Shared memory holds
// the tile row by row (pitch W | 1, so that a column walk is free of bank
// conflicts), the Q rows innermost when the members' narrow sides run along
// Q, else the P rows.  Destination-wide: the members gather their elements
// into the zeroed tile, which is then written as whole rows (columns no member
// covers are structural zeros or padding of the operand).  Source-wide: whole
// rows are read, then each member scatters its columns.  Each member walks its
// elements in the order of its narrow-side strides, so that side coalesces too.
__device__ void copy_band(const CopyTask* __restrict__ tasks, int h, int tile, double* const* __restrict__ slots,
                          double* buf, tnx_band::Member* mem, int* pre) {
  using namespace tnx_band;
  const CopyTask& H = tasks[h];
  const int nt = H.rank;
  const int EP = H.shape[0], EQ = H.shape[1], W = H.shape[2], TP = H.shape[3], TQ = H.shape[4];
  const bool dwide = H.shape[5] != 0, qin = H.shape[6] != 0;
  const int Wp = W | 1;
  const int ntq = (EQ + TQ - 1) / TQ;
  const int tp = tile / ntq, tq = tile - tp * ntq;
  const int p0 = tp * TP, q0 = tq * TQ;
  const int tP = min(TP, EP - p0), tQ = min(TQ, EQ - q0);
  const int wP = qin ? tQ * Wp : Wp, wQ = qin ? Wp : tP * Wp;
  if ((int)threadIdx.x < nt) mem[threadIdx.x] = stage(tasks[h + 1 + threadIdx.x], dwide, p0, q0, tP, tQ, wP, wQ);
  const int rows = tP * tQ;
  const long long XP = H.sstride[0], XQ = H.sstride[1];
  const long long wbase = (dwide ? H.dst_off : H.src_off) + (long long)p0 * XP + (long long)q0 * XQ;
  double* wptr = slots[dwide ? H.dst_slot : H.src_slot] + wbase;
  const float invW = 1.0f / (float)W, invR = 1.0f / (float)(qin ? tQ : tP);
  // wide row r of the tile -> offset of its first element on the wide side
  auto rowoff = [&](int r) -> long long {
    int p, q;
    if (qin) {
      p = qdiv(r, tQ, invR);
      q = r - p * tQ;
    } else {
      q = qdiv(r, tP, invR);
      p = r - q * tP;
    }
    return (long long)p * XP + (long long)q * XQ;
  };
  if (dwide) {
    for (int i = threadIdx.x; i < rows * Wp; i += CT) buf[i] = 0.0;
  } else {
    // kUnroll loads in flight per thread before their shared-memory stores
    for (int e0 = threadIdx.x; e0 < rows * W; e0 += CT * kUnroll) {
      double v[kUnroll];
      int so[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int e = e0 + u * CT;
        so[u] = -1;
        if (e < rows * W) {
          const int r = qdiv(e, W, invW), c = e - r * W;
          so[u] = r * Wp + c;
          v[u] = __ldg(wptr + rowoff(r) + c);
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        if (so[u] >= 0) buf[so[u]] = v[u];
    }
  }
  __syncthreads();
  prefix(mem, nt, pre);
  __syncthreads();
  if (dwide) move<CT, true>(mem, pre, nt, buf, slots);
  else move<CT, false>(mem, pre, nt, buf, slots);
  if (dwide) {
    __syncthreads();
    for (int e = threadIdx.x; e < rows * W; e += CT) {
      const int r = qdiv(e, W, invW), c = e - r * W;
      wptr[rowoff(r) + c] = buf[r * Wp + c];
    }
  }
}

// Source / destination offsets of in-task element i: decompose i over the
// legs (last leg fastest).
__device__ __forceinline__ void offsets(const CopyTask& t, int i, int& so, int& dof) {
  so = 0;
  dof = 0;
#pragma unroll
  for (int l = TNX_MAXR - 1; l >= 0; --l) {
    if (l < t.rank) {
      const int q = fdiv(i, t.magic[l], t.shift[l]);
      const int rem = i - q * t.shape[l];
      i = q;
      so += rem * t.sstride[l];
      dof += rem * t.dstride[l];
    }
  }
}

// Elements [e0, e0 + n) of one task (n <= EPT): one decomposition, then steps
// along the innermost leg; a carry into the next leg re-decomposes.
constexpr int EPT = 2;

template <bool SCALED>
__device__ __forceinline__ void copy_run(const CopyTask& t, const double* src, double* dst, int e0, int n,
                                         double scale, double* vdst) {
  int so, dof;
  offsets(t, e0, so, dof);
  const int last = t.rank - 1;
  const int ext = t.shape[last];
  int pos = e0 - fdiv(e0, t.magic[last], t.shift[last]) * ext;
  const int ss = t.sstride[last], ds = t.dstride[last];
  double v[EPT];
  int d[EPT], sv[EPT];
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    if (j < n) {
      v[j] = src ? __ldg(src + so) : 0.0;
      d[j] = dof;
      sv[j] = so;
      if (++pos == ext) {
        pos = 0;
        offsets(t, e0 + j + 1, so, dof);
      } else {
        so += ss;
        dof += ds;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    if (j < n) {
      if (SCALED) {
        const double y = v[j] * scale;
        dst[d[j]] = y;
        if (vdst) vdst[sv[j]] = y;
      } else {
        dst[d[j]] = v[j];
      }
    }
  }
}

// Scaled relayout (the normalising step of a Lanczos iteration, fused with the
// next apply's relayout of the vector): every task reads src (instead of its
// source slot) times *inv.  vdst = src * *inv is written by blocks past the
// chunks over vn contiguous entries, or, when the tasks read every entry once
// (full), by the tasks themselves from the product they store.  Nothing runs
// once the solve has stopped.
struct ScaleArgs {
  const double* src;
  double* vdst;
  int64_t vn;
  int nchunks;
  int full;
  const double* inv;
  const int32_t* state;
};

// chunk = (first task, first element, number of tasks, number of elements).
// One task: its elements [first, first + count), EPT consecutive ones per
// thread.  Several (small) tasks: all their elements, back to back; the
// chunk's descriptors are staged in shared memory and each thread finds its
// task by binary search over their starts.  Task count -1 marks one 32 x 32
// tile of a transposing task, -2 one tile of a band.
template <bool SCALED>
__global__ void __launch_bounds__(CT) copy_kernel(const CopyTask* __restrict__ tasks, const int4* __restrict__ chunks,
                                                  double* const* __restrict__ slots, ScaleArgs sa) {
  tnx_grid_dependency();
  double scale = 1.0;
  if (SCALED) {
    if (*(volatile const int32_t*)(sa.state + 1) != 0) return;   // the solve has stopped
    scale = *sa.inv;
    if ((int)blockIdx.x >= sa.nchunks) {
      const int64_t stride = (int64_t)(gridDim.x - sa.nchunks) * CT;
      for (int64_t i = (int64_t)(blockIdx.x - sa.nchunks) * CT + threadIdx.x; i < sa.vn; i += stride)
        sa.vdst[i] = sa.src[i] * scale;
      return;
    }
  }
  // packed tasks | transposing tile | band tile (members, then the staged rows)
  constexpr int kPack = TNX_COPY_PACK * (int)sizeof(CopyTask);
  constexpr int kBand = TNX_BAND_MAXM * (int)sizeof(tnx_band::Member) + TNX_BAND_CAP * 8;
  constexpr int kRaw = kPack > kBand ? kPack : kBand;
  static_assert(32 * 33 * 8 <= kRaw, "shared memory of the transposing tile");
  __shared__ __align__(16) unsigned char raw[kRaw];
  __shared__ int sstart[TNX_BAND_MAXM > TNX_COPY_PACK ? TNX_BAND_MAXM + 1 : TNX_COPY_PACK + 1];
  CopyTask* st = (CopyTask*)raw;
  const int4 ch = chunks[blockIdx.x];
  if (ch.z == -1) {
    copy_transpose<SCALED>(tasks[ch.x], ch.y, slots, (double (*)[33])raw, sa.src, scale,
                           SCALED && sa.full ? sa.vdst : nullptr);
    return;
  }
  if (!SCALED && ch.z == -2) {
    copy_band(tasks, ch.x, ch.y, slots, (double*)(raw + TNX_BAND_MAXM * sizeof(tnx_band::Member)), (tnx_band::Member*)raw, sstart);
    return;
  }
  if (ch.z == 1) {
    {
      const int* g = (const int*)(tasks + ch.x);
      int* sm = (int*)st;
      for (int i = threadIdx.x; i < (int)(sizeof(CopyTask) / 4); i += CT) sm[i] = g[i];
    }
    __syncthreads();
    const CopyTask& t = st[0];
    const double* src = SCALED ? sa.src + t.src_off : (t.src_slot >= 0 ? slots[t.src_slot] + t.src_off : nullptr);
    double* dst = slots[t.dst_slot] + t.dst_off;
    const int end = ch.y + ch.w;
    double* vd = SCALED && sa.full ? sa.vdst + t.src_off : nullptr;
    for (int e = ch.y + threadIdx.x * EPT; e < end; e += CT * EPT)
      copy_run<SCALED>(t, src, dst, e, min(EPT, end - e), scale, vd);
    return;
  }
  // several small tasks
  const int nt = ch.z;
  {
    const int words = (int)(sizeof(CopyTask) / 4) * nt;
    const int* g = (const int*)(tasks + ch.x);
    int* sm = (int*)st;
    for (int i = threadIdx.x; i < words; i += CT) sm[i] = g[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int k = 0; k < nt; ++k) {
      sstart[k] = acc;
      acc += (int)st[k].nelem;
    }
    sstart[nt] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ch.w; e += CT) {
    int lo = 0, hi = nt;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (sstart[mid] <= e) lo = mid; else hi = mid;
    }
    const CopyTask& t = st[lo];
    const double* src = SCALED ? sa.src + t.src_off : (t.src_slot >= 0 ? slots[t.src_slot] + t.src_off : nullptr);
    int so, dof;
    offsets(t, e - sstart[lo], so, dof);
    const double x = src ? __ldg(src + so) : 0.0;
    if (SCALED) {
      const double y = x * scale;
      slots[t.dst_slot][t.dst_off + dof] = y;
      if (sa.full) sa.vdst[t.src_off + so] = y;
    } else {
      slots[t.dst_slot][t.dst_off + dof] = x;
    }
  }
}

}  // namespace

cudaError_t tnx_launch_copy(const CopyTask* tasks, const int4* chunks, int nchunks, double* const* slots,
                            cudaStream_t st) {
  if (nchunks <= 0) return cudaSuccess;
  {
    const cudaError_t le = tnx_launch(copy_kernel<false>, dim3(nchunks), dim3(CT), 0, st, tasks, chunks, slots,
                                      ScaleArgs{nullptr, nullptr, 0, nchunks, 0, nullptr, nullptr});
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  return cudaGetLastError();
}

cudaError_t tnx_launch_copy_scaled(const CopyTask* tasks, const int4* chunks, int nchunks, double* const* slots,
                                   const double* src, double* vdst, int64_t vn, int full, const double* inv,
                                   const int32_t* state, cudaStream_t st) {
  if (nchunks < 0 || vn < 0 || (full && nchunks == 0 && vn > 0)) return cudaErrorInvalidValue;
  const int64_t vb = full ? 0 : std::max<int64_t>(std::min<int64_t>((vn + CT * 4 - 1) / (CT * 4), 1216), 1);
  const int64_t grid = (int64_t)nchunks + vb;
  if (grid == 0) return cudaSuccess;
  if (grid > INT32_MAX) return cudaErrorInvalidValue;
  {
    const cudaError_t le = tnx_launch(copy_kernel<true>, dim3((unsigned)grid), dim3(CT), 0, st, tasks, chunks, slots,
                                      ScaleArgs{src, vdst, vn, nchunks, full, inv, state});
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  return cudaGetLastError();
}
