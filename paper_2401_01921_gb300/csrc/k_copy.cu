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
// through shared memory instead, so both sides coalesce.  Index arithmetic is
// 32-bit inside a task, and an index is split over the legs with
// multiply-high divisions by the leg extents (constants the planner
// precomputes) instead of hardware integer divisions.
#include "tnx_internal.h"

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
__device__ void copy_transpose(const CopyTask& t, int tile, double* const* __restrict__ slots) {
  __shared__ double sm[32][33];
  const int r = t.rank, S = t.tleg;
  const int ncols = t.shape[S];
  const int nrows = (int)(t.nelem / ncols);
  const int nct = (ncols + 31) >> 5;
  const int r0 = (tile / nct) << 5, c0 = (tile % nct) << 5;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double* src = t.src_slot >= 0 ? slots[t.src_slot] + t.src_off : nullptr;
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
      sm[rr][lane] = src ? __ldg(src + so + c * t.sstride[S]) : 0.0;
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

__device__ __forceinline__ void copy_run(const CopyTask& t, const double* src, double* dst, int e0, int n) {
  int so, dof;
  offsets(t, e0, so, dof);
  const int last = t.rank - 1;
  const int ext = t.shape[last];
  int pos = e0 - fdiv(e0, t.magic[last], t.shift[last]) * ext;
  const int ss = t.sstride[last], ds = t.dstride[last];
  double v[EPT];
  int d[EPT];
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    if (j < n) {
      v[j] = src ? __ldg(src + so) : 0.0;
      d[j] = dof;
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
  for (int j = 0; j < EPT; ++j)
    if (j < n) dst[d[j]] = v[j];
}

// chunk = (first task, first element, number of tasks, number of elements).
// One task: its elements [first, first + count), EPT consecutive ones per
// thread.  Several (small) tasks: all their elements, back to back; the
// chunk's descriptors are staged in shared memory and each thread finds its
// task by binary search over their starts.  A negative task count marks one
// 32 x 32 tile of a transposing task.
__global__ void __launch_bounds__(CT) copy_kernel(const CopyTask* __restrict__ tasks, const int4* __restrict__ chunks,
                                                  double* const* __restrict__ slots) {
  tnx_grid_dependency();
  __shared__ CopyTask st[TNX_COPY_PACK];
  __shared__ int sstart[TNX_COPY_PACK + 1];
  const int4 ch = chunks[blockIdx.x];
  if (ch.z < 0) {
    copy_transpose(tasks[ch.x], ch.y, slots);
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
    const double* src = t.src_slot >= 0 ? slots[t.src_slot] + t.src_off : nullptr;
    double* dst = slots[t.dst_slot] + t.dst_off;
    const int end = ch.y + ch.w;
    for (int e = ch.y + threadIdx.x * EPT; e < end; e += CT * EPT) copy_run(t, src, dst, e, min(EPT, end - e));
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
    const double* src = t.src_slot >= 0 ? slots[t.src_slot] + t.src_off : nullptr;
    int so, dof;
    offsets(t, e - sstart[lo], so, dof);
    slots[t.dst_slot][t.dst_off + dof] = src ? __ldg(src + so) : 0.0;
  }
}

}  // namespace

cudaError_t tnx_launch_copy(const CopyTask* tasks, const int4* chunks, int nchunks, double* const* slots,
                            cudaStream_t st) {
  if (nchunks <= 0) return cudaSuccess;
  {
    const cudaError_t le = tnx_launch(copy_kernel, dim3(nchunks), dim3(CT), 0, st, tasks, chunks, slots);
    if (le != cudaSuccess) return le;
  }
  tnx_note_launch(1);
  return cudaGetLastError();
}
