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
// in the destination.  Threads walk destination order, so stores coalesce;
// when the source is contiguous along the same leg the loads coalesce too.
#include "tnx_internal.h"

namespace {

constexpr int CT = 256;

__device__ __forceinline__ int find_task(const int64_t* start, int n, int64_t e) {
  int lo = 0, hi = n;   // start[lo] <= e < start[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(start + mid) <= e) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(CT) copy_kernel(const CopyTask* __restrict__ tasks,
                                                  const int64_t* __restrict__ start, int ntasks, int64_t total,
                                                  double* const* __restrict__ slots) {
  for (int64_t e = (int64_t)blockIdx.x * CT + threadIdx.x; e < total; e += (int64_t)gridDim.x * CT) {
    const int ti = find_task(start, ntasks, e);
    const CopyTask& t = tasks[ti];
    int64_t i = e - __ldg(start + ti);
    int64_t so = t.src_off, dof = t.dst_off;
    for (int l = t.rank - 1; l >= 0; --l) {
      const int s = t.shape[l];
      const int64_t q = i / s;
      const int64_t r = i - q * s;
      i = q;
      so += r * t.sstride[l];
      dof += r * t.dstride[l];
    }
    double v = 0.0;
    if (t.src_slot >= 0) v = __ldg(slots[t.src_slot] + so);
    slots[t.dst_slot][dof] = v;
  }
}

}  // namespace

cudaError_t tnx_launch_copy(const CopyTask* tasks, const int64_t* elem_start, int ntasks, int64_t total,
                            double* const* slots, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  int64_t blocks = (total + CT - 1) / CT;
  const int64_t cap = 152 * 16;
  if (blocks > cap) blocks = cap;
  copy_kernel<<<(int)blocks, CT, 0, st>>>(tasks, elem_start, ntasks, total, slots);
  tnx_note_launch(1);
  return cudaGetLastError();
}
