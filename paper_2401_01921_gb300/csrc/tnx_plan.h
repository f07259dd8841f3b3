// Host-only plan structures shared by the planner (tnx_network.cpp) and the
// split-precision planner (tnx_split.cpp).
#pragma once

#include <algorithm>
#include <cstring>

#include "tnx_host.h"

struct NetTensor {
  std::string name;
  std::vector<std::string> labels;
  tnx_tensor* t = nullptr;
  std::vector<int> perm;   // perm[j] = leg of t realising blueprint leg j
};

struct TreeNode {
  int leaf = -1, l = -1, r = -1;
};

struct OpView {
  std::vector<BondD> bonds;
  std::vector<std::string> labels;
  int64_t nblk = 0;
  std::vector<int32_t> qn;      // nblk * rank, lexicographic
  std::vector<int64_t> base;    // nblk
  std::vector<int64_t> stride;  // nblk * rank
  // GEMM outputs only: legs [0, nrow) are row legs of a row-major matrix, and
  // per block the offset of its first row's start and the row length
  int nrow = -1;
  std::vector<int64_t> rowstart, rowld;
  bool skinny_out = false;      // output of a step whose groups all have K <= 16
  int slot = -1;
  int rank() const { return (int)bonds.size(); }
};

struct TaskList {
  CopyTask* d = nullptr;
  int4* chunks = nullptr;
  int nchunks = 0;
  int n = 0;
  int64_t total = 0;
  std::vector<CopyTask> h;      // host copies (batched plans merge them)
  std::vector<int4> hchunks;
};

struct StepPlan {
  OpView A, B, C;
  uint64_t leavesA = 0, leavesB = 0;   // network tensors feeding each operand (bit i = tensor i)
  std::vector<int> ka, kb, fa, fb;
  int G = 0;
  std::vector<int32_t> charges;
  std::vector<int64_t> mkn, amap, bmap;
  std::vector<int64_t> ldK, offA, offB, offC;
  double flops = 0;
  int nsym = 0;
  int slotA = -1, slotB = -1, slotC = -1;
  TaskList copyA, copyB;
  GemmGroup* dG = nullptr;
  GemmTile* dT = nullptr;
  int ntiles = 0;
  GemmTile* dTs = nullptr;      // skinny (K <= 16) tiles, FP64 in every precision
  int nstiles_skinny = 0;
  std::vector<GemmGroup> hG;    // host copies
  std::vector<GemmTile> hT, hTs;
  std::vector<char> skinny;     // per group
  double flops_skinny = 0;      // useful flops of the skinny groups
  // split precision
  int slotSA = -1, slotSB = -1, slotEA = -1, slotEB = -1;
  int slotKX = -1;              // K balancing words (int32, whole K tiles per group)
  KexpJob* dKJ = nullptr;       // their jobs (one per split group) and work items
  int nkj = 0;
  int4* dKI = nullptr;
  int64_t nki = 0;
  std::vector<KexpJob> hKJ;     // host copy (batched plans merge them)
  struct Jobs {             // one slicing launch: its jobs and work items
    SliceJob* d = nullptr;
    int n = 0;
    int2* items = nullptr;      // (job, first 8-row group) per CTA work item
    int64_t nitems = 0;
    int64_t elems = 0;
    std::vector<SliceJob> h;    // host copies (batched plans merge them)
  } jobsAll, jobsA, jobsB;
  int64_t slice_elems = 0;      // packed elements that get sliced (split precision)
  SplitGroup* dSG = nullptr;
  GemmTile* dST = nullptr;
  int nstiles = 0;
  int split_tn = 64;            // tile width of the split GEMM (B slices are tiled to match)
  int split_grid = 0;           // CTAs of the split GEMM; dST holds its per-CTA schedule (holes: group -1)
  bool split_fold = false;      // its epilogue writes the network's output (the folded output relayout)
  int split_kmax = 0;           // largest K of its split groups
  std::vector<SplitGroup> hSG;  // host copies
  std::vector<GemmTile> hST;    // tiles longest K first, no holes (batched plans merge them)
  // fused skinny step (k_fused.cu): one launch replaces the relayout of A, the
  // skinny product and (when fscatter is set) the next step's relayout of C
  FusedTile* dFT = nullptr;
  FusedCol* dFC = nullptr;
  int nftiles = 0;
  int fkp = 0, fnp = 0;
  bool fscatter = false;               // output stored into the next step's operand
  bool skipA = false, skipB = false;   // this step's operand relayout is done by a fused step
  std::vector<FusedTile> hFT;
  std::vector<FusedCol> hFC;
};

// A captured CUDA graph plus the profiler events recorded inside it.
struct GraphRec {
  cudaGraphExec_t exec = nullptr;
  std::vector<ProfRec> recs;
  long long nlaunch = 0;          // kernel launches inside the graph (counted per replay)
  uint32_t prof = 0;              // profiled classes when captured
  ~GraphRec() {
    if (exec) cudaGraphExecDestroy(exec);
    for (auto& r : recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
  }
};

struct Plan {
  tnx_ctx* ctx = nullptr;
  uint64_t serial = 0;            // unique per plan (cache key of dependent graphs)
  std::unique_ptr<GraphRec> apply_graph;
  int eager_applies = 0;          // applies run without a graph (the first one)
  std::vector<std::unique_ptr<DevBuf>> bufs;
  std::vector<double*> h_slots, h_slots_dev;   // wanted / last uploaded
  double** d_slots = nullptr;
  int nin = 0, out_slot = 0;
  std::vector<StepPlan> steps;
  std::vector<BondD> out_bonds;
  std::vector<std::string> out_labels;
  TaskList fin;
  bool fin_folded = false;       // the last split product writes the output itself (fin unused)
  int prec = TNX_PREC_F64;
  int nslice = 6, beta = 7;
  bool narrow_tiles = true;       // from the network (a batch needs the same tile width in every plan)
  int32_t* d_status = nullptr;
  std::string key;
  std::string order;
  ~Plan() = default;

  // Sizing pass (dry): the planner runs as usual (the matching kernel included)
  // but plan buffers are only counted, at stand-in addresses nothing reads.
  bool dry = false;
  size_t dry_bytes = 0;
  uintptr_t dry_next = 4096;
  void* dry_take(size_t n) {
    dry_bytes += n;
    void* p = (void*)dry_next;
    dry_next += (n + 255) & ~(size_t)255;
    return p;
  }
  template <class T>
  T* upload(const std::vector<T>& v) {
    size_t n = std::max<size_t>(v.size(), 1) * sizeof(T);
    if (dry) return (T*)dry_take(n);
    bufs.emplace_back(new DevBuf(ctx, n));
    if (!v.empty()) CUDA_CHECK(cudaMemcpyAsync(bufs.back()->p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return (T*)bufs.back()->p;
  }
  void* alloc_zero(size_t bytes) {
    if (dry) return dry_take(std::max<size_t>(bytes, 256));
    bufs.emplace_back(new DevBuf(ctx, std::max<size_t>(bytes, 256)));
    CUDA_CHECK(cudaMemsetAsync(bufs.back()->p, 0, std::max<size_t>(bytes, 256), ctx->stream));
    return bufs.back()->p;
  }
  std::vector<int64_t> slot_elems;   // size of each slot's buffer, in doubles
  int new_slot(void* p, int64_t elems) {
    h_slots.push_back((double*)p);
    slot_elems.push_back(elems);
    return (int)h_slots.size() - 1;
  }
};

struct tnx_network {
  tnx_ctx* ctx = nullptr;
  std::vector<NetTensor> ts;
  std::vector<std::string> tout;
  std::vector<TreeNode> tree;
  int root = -1;
  int optimal = 0;                 // 0 explicit order, 1 dense-cost search, 2 block-sparse-cost search
  bool narrow_tiles = true;        // split GEMM steps with few tiles may use 32-wide tiles
  int prec = TNX_PREC_F64;
  std::string order_dims_key;      // dims for which the optimal tree was computed
  std::string sized_key;           // plan key of the last sizing pass, and its bytes
  size_t sized_bytes = 0;
  std::unique_ptr<Plan> plan;
  std::unique_ptr<struct LanczosCache> lanczos;
  ~tnx_network();
};


// split-precision planning and launch (tnx_split.cpp)
void tnx_build_split_parts(Plan& p, StepPlan& s);
// balance: K-balanced slicing (A's column exponents), recomputed when A is
std::vector<int4> tnx_kexp_items(const std::vector<KexpJob>& jobs);
void tnx_enqueue_split(Plan& p, StepPlan& s, cudaStream_t st, bool needA, bool needB, bool balance);
std::vector<int2> tnx_slice_schedule(std::vector<SliceJob>& jobs);
std::vector<int2> tnx_tf32_schedule(std::vector<SliceJob>& jobs);

// relayout chunks (tnx_network.cpp)
void tnx_make_copy_chunks(const std::vector<CopyTask>& tasks, std::vector<int4>& chunks);
std::vector<CopyTask> tnx_unband_tasks(const std::vector<CopyTask>& tasks);

// enqueue helpers shared by the C-ABI, the batch and the serving modules (tnx_network.cpp)
Plan* tnx_ensure_plan(tnx_network* net);
void tnx_apply_enqueue(tnx_network* net, tnx_tensor* out, cudaStream_t st);
void tnx_lanczos_enqueue(tnx_network* net, int slot, tnx_tensor* v0, int nsteps, tnx_tensor* evec, cudaStream_t st,
                         double* host_out);
int tnx_network_slot(tnx_network* net, const char* name);
size_t tnx_network_resident_bytes(tnx_network* net);
// Device bytes the network's plan holds (its current plan, or a sizing pass
// that allocates nothing but the matching kernel's temporaries), and the bytes
// of a Lanczos workspace for n-element vectors and nsteps steps.
size_t tnx_network_plan_bytes(tnx_network* net);
size_t tnx_lanczos_workspace_bytes(int64_t n, int nsteps);
// Bytes of the network's current Lanczos workspace (0 if none).
size_t tnx_network_lanczos_bytes(tnx_network* net);
void tnx_network_evict(tnx_network* net);
