// Host side of the C-ABI: contexts, bonds, block-sparse tensors and the
// parts of the network contraction that are not kernels.
//
// Follows arXiv 2401.01921:
//   Sec. 6.1-6.3  symmetries, bonds with quantum numbers, zero-flux block
//                 enumeration in block-index (lexicographic Qn) order;
//   Sec. 6.2.2    bond combine (grouped, ascending);
//   Sec. 6.3      scalar multiply allowed, scalar add refused on symmetric tensors.
// The network planner / executor is in tnx_network.cpp.
#include "tnx_host.h"

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <numeric>
#include <cstdlib>

// ------------------------------------------------------------------ context
void* tnx_ctx::dalloc(size_t n) {
  if (n == 0) n = 256;
  n = (n + 255) & ~size_t(255);
  void* p = nullptr;
  if (alloc) {
    p = alloc(n, user);
  } else {
    cudaError_t e = cudaMallocAsync(&p, n, stream);
    if (e != cudaSuccess) p = nullptr;
  }
  if (!p) fail(TNX_ERR_OOM, "device allocation of " + std::to_string(n) + " bytes failed");
  return p;
}

void tnx_ctx::dfree(void* p, size_t n) {
  if (!p) return;
  if (n == 0) n = 256;
  n = (n + 255) & ~size_t(255);
  if (fre) fre(p, n, user);
  else if (!alloc) cudaFreeAsync(p, stream);
}

DevBuf::DevBuf(tnx_ctx* c, size_t n) : ctx(c), bytes(n) { p = c->dalloc(n); }
DevBuf::~DevBuf() { if (ctx && p) ctx->dfree(p, bytes); }

// ----------------------------------------------------------------- counters
static std::atomic<long long> g_launches{0};
// While a thread captures a CUDA graph, its launches are counted into the
// graph's record instead (they run when the graph is launched).
static thread_local long long* t_capture_count = nullptr;

void tnx_note_launch(long long n) {
  if (t_capture_count) *t_capture_count += n;
  else g_launches += n;
}

void tnx_count_into(long long* c) { t_capture_count = c; }

extern "C" tnx_status tnx_kernel_launches(int64_t* n) {
  if (!n) return TNX_ERR_ARG;
  *n = g_launches.load();
  return TNX_OK;
}

cudaEvent_t tnx_ctx::get_event() {
  if (!event_pool.empty()) {
    cudaEvent_t e = event_pool.back();
    event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CUDA_CHECK(cudaEventCreate(&e));
  return e;
}

// Inside a stream capture an event must be recorded as an external event node
// to carry a timestamp when the graph runs.
static void record_event(tnx_ctx* c, cudaEvent_t e, cudaStream_t st) {
  if (c->capture_recs) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  else cudaEventRecord(e, st);
}

ProfScope::ProfScope(tnx_ctx* c_, cudaStream_t s_, int cls_, double work_) : c(c_), st(s_), cls(cls_), work(work_) {
  if ((c->prof >> cls) & 1u) {
    if (c->capture_recs) cudaEventCreate(&a);
    else a = c->get_event();
    record_event(c, a, st);
  }
}

ProfScope::~ProfScope() {
  if (!a) return;
  cudaEvent_t b;
  if (c->capture_recs) cudaEventCreate(&b);
  else b = c->get_event();
  record_event(c, b, st);
  if (c->capture_recs) c->capture_recs->push_back(ProfRec{a, b, cls, work});
  else c->prof_pending.push_back(ProfRec{a, b, cls, work});
}

void prof_accumulate(tnx_ctx* c, const std::vector<ProfRec>& recs) {
  for (auto& r : recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.cls] += ms;
      c->prof_n[r.cls] += 1;
      c->prof_work[r.cls] += r.work;
    } else {
      cudaGetLastError();   // leave no stale error behind for the caller
    }
  }
}

static void prof_drain(tnx_ctx* c) {
  for (auto& r : c->prof_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.cls] += ms;
      c->prof_n[r.cls] += 1;
      c->prof_work[r.cls] += r.work;
    } else {
      cudaGetLastError();
    }
    c->event_pool.push_back(r.a);
    c->event_pool.push_back(r.b);
  }
  c->prof_pending.clear();
}

extern "C" tnx_status tnx_profile_classes(tnx_ctx* ctx, uint32_t class_mask) {
  if (!ctx) return TNX_ERR_ARG;
  return tnx_guard(ctx, [&] {
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    prof_drain(ctx);
    for (int i = 0; i < TNX_KC_COUNT; ++i) ctx->prof_ms[i] = 0, ctx->prof_n[i] = 0, ctx->prof_work[i] = 0;
    ctx->prof = class_mask & (((1u << TNX_KC_COUNT) - 1u) | TNX_PROF_LAST_APPLY);
    if (!(ctx->prof & ((1u << TNX_KC_COUNT) - 1u))) ctx->prof = 0;
  });
}

extern "C" tnx_status tnx_profile_enable(tnx_ctx* ctx, int enable) {
  return tnx_profile_classes(ctx, enable ? (1u << TNX_KC_COUNT) - 1u : 0u);
}

extern "C" tnx_status tnx_profile_read(tnx_ctx* ctx, double* ms, int64_t* launches, double* work) {
  if (!ctx) return TNX_ERR_ARG;
  return tnx_guard(ctx, [&] {
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    prof_drain(ctx);
    for (int i = 0; i < TNX_KC_COUNT; ++i) {
      if (ms) ms[i] = ctx->prof_ms[i];
      if (launches) launches[i] = ctx->prof_n[i];
      if (work) work[i] = ctx->prof_work[i];
    }
  });
}

static tnx_status set_err(tnx_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

tnx_status tnx_guard(tnx_ctx* ctx, const std::function<void()>& f) {
  try {
    if (ctx) {
      int dev = -1;
      if (cudaGetDevice(&dev) == cudaSuccess && dev != ctx->device) cudaSetDevice(ctx->device);
    }
    f();
    return TNX_OK;
  } catch (const TnxError& e) {
    if (e.code == TNX_ERR_CUDA) cudaGetLastError();
    return set_err(ctx, e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return set_err(ctx, TNX_ERR_OOM, "host out of memory");
  } catch (const std::exception& e) {
    return set_err(ctx, TNX_ERR_ARG, e.what());
  }
}

extern "C" const char* tnx_last_error(const tnx_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" const char* tnx_version(void) { return "tnx 1.0"; }

extern "C" tnx_status tnx_ctx_create(int device, void* stream, tnx_alloc_fn alloc, tnx_free_fn fre, void* user,
                                     tnx_ctx** out) {
  if (!out) return TNX_ERR_ARG;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return TNX_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return TNX_ERR_CUDA;
  auto* c = new tnx_ctx();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  c->alloc = alloc;
  c->fre = fre;
  c->user = user;
  {
    const char* ng = getenv("TNX_NO_GRAPHS");
    c->use_graphs = !(ng && *ng && *ng != '0');
  }
  tnx_status s = tnx_guard(c, [&] {
    c->scratch = new DevBuf(c, 64 * 1024);
    c->d_status = (int32_t*)((char*)c->scratch->p + 63 * 1024);
    CUDA_CHECK(cudaMemsetAsync(c->d_status, 0, 64, c->stream));
    c->pinned = nullptr;
    CUDA_CHECK(cudaMallocHost(&c->pinned, 4096));
  });
  if (s != TNX_OK) {
    delete c;
    return s;
  }
  *out = c;
  return TNX_OK;
}

extern "C" tnx_status tnx_ctx_destroy(tnx_ctx* ctx) {
  if (!ctx) return TNX_ERR_ARG;
  cudaStreamSynchronize(ctx->stream);
  prof_drain(ctx);
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  delete ctx->scratch;
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
  return TNX_OK;
}

void check_device_status(tnx_ctx* ctx) {
  int32_t* h = (int32_t*)ctx->pinned + 512;
  CUDA_CHECK(cudaMemcpyAsync(h, ctx->d_status, 4, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
  if (*h != 0) {
    const int code = *h;
    CUDA_CHECK(cudaMemsetAsync(ctx->d_status, 0, 4, ctx->stream));
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    fail(TNX_ERR_TIMEOUT, "a bounded device wait ran out (site " + std::to_string(code) + ")");
  }
}

extern "C" tnx_status tnx_sync(tnx_ctx* ctx) {
  if (!ctx) return TNX_ERR_ARG;
  return tnx_guard(ctx, [&] {
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    check_device_status(ctx);
  });
}

// -------------------------------------------------------------------- bonds
int32_t BondD::signed_q(int s, int c) const {
  int32_t q = qn[(size_t)s * nsym + c];
  if (dir == TNX_BD_OUT) q = -q;
  if (kinds[c] == TNX_ZN) q = ((q % zn[c]) + zn[c]) % zn[c];
  return q;
}

bool BondD::same_syms(const BondD& o) const { return nsym == o.nsym && kinds == o.kinds && zn == o.zn; }

bool BondD::operator==(const BondD& o) const {
  return dir == o.dir && same_syms(o) && nsec == o.nsec && qn == o.qn && deg == o.deg;
}

void BondD::finish() {
  off.assign(nsec + 1, 0);
  for (int s = 0; s < nsec; ++s) off[s + 1] = off[s] + deg[s];
  dim = off[nsec];
}

std::string BondD::key() const {
  std::string k = std::to_string(dir) + "|" + std::to_string(nsym) + "|";
  for (int c = 0; c < nsym; ++c) k += std::to_string(kinds[c]) + ":" + std::to_string(zn[c]) + ",";
  k += "|";
  for (int s = 0; s < nsec; ++s) {
    for (int c = 0; c < nsym; ++c) k += std::to_string(qn[(size_t)s * nsym + c]) + ",";
    k += ":" + std::to_string(deg[s]) + ";";
  }
  return k;
}

// Sec. 7: contracted bonds: equal dimension; for symmetric bonds opposite
// directions and identical sectors (charges and degeneracies).
void check_contractible(const BondD& a, const BondD& b, const std::string& label) {
  if (a.dim != b.dim) fail(TNX_ERR_BOND_MISMATCH, "dimension mismatch on label '" + label + "'");
  if (!a.same_syms(b)) fail(TNX_ERR_BOND_MISMATCH, "symmetry mismatch on label '" + label + "'");
  if (a.nsym > 0) {
    if (a.dir == TNX_BD_REG || b.dir == TNX_BD_REG || a.dir != -b.dir)
      fail(TNX_ERR_BOND_MISMATCH, "direction mismatch on label '" + label + "' (an IN leg meets an OUT leg)");
    if (a.qn != b.qn || a.deg != b.deg)
      fail(TNX_ERR_BOND_MISMATCH, "charge sectors differ on label '" + label + "'");
  } else if (a.deg != b.deg) {
    fail(TNX_ERR_BOND_MISMATCH, "dimension mismatch on label '" + label + "'");
  }
}

extern "C" tnx_status tnx_bond_create(tnx_ctx* ctx, int dir, int nsym, const int* kinds, const int* zn, int nsec,
                                      const int32_t* qnums, const int64_t* degs, tnx_bond** out) {
  return tnx_guard(ctx, [&] {
    if (!ctx || !out || nsec < 1 || !degs || nsym < 0 || nsym > TNX_MAXSYM) fail(TNX_ERR_ARG, "bad bond arguments");
    if (nsym > 0 && (!kinds || !qnums)) fail(TNX_ERR_ARG, "symmetric bond needs kinds and qnums");
    if (nsym == 0 && (dir != TNX_BD_REG || nsec != 1)) fail(TNX_ERR_ARG, "a plain bond is REGULAR with one sector");
    if (nsym > 0 && dir != TNX_BD_IN && dir != TNX_BD_OUT) fail(TNX_ERR_ARG, "a symmetric bond is IN or OUT");
    auto* b = new tnx_bond();
    b->ctx = ctx;
    BondD& d = b->b;
    d.dir = dir;
    d.nsym = nsym;
    d.nsec = nsec;
    for (int c = 0; c < nsym; ++c) {
      if (kinds[c] != TNX_U1 && kinds[c] != TNX_ZN) { delete b; fail(TNX_ERR_ARG, "unknown symmetry kind"); }
      if (kinds[c] == TNX_ZN && (!zn || zn[c] < 2)) { delete b; fail(TNX_ERR_ARG, "Z_n needs n >= 2"); }
      if (kinds[c] == TNX_ZN && zn[c] > TNX_QMAX) { delete b; fail(TNX_ERR_UNSUPPORTED, "Z_n modulus above 2^24"); }
      d.kinds.push_back(kinds[c]);
      d.zn.push_back(kinds[c] == TNX_ZN ? zn[c] : 0);
    }
    for (int s = 0; s < nsec; ++s) {
      if (degs[s] < 1) { delete b; fail(TNX_ERR_ARG, "degeneracy must be >= 1"); }
      d.deg.push_back(degs[s]);
      for (int c = 0; c < nsym; ++c) {
        int32_t q = qnums[(size_t)s * nsym + c];
        if (d.kinds[c] == TNX_ZN) q = ((q % d.zn[c]) + d.zn[c]) % d.zn[c];
        if (q > TNX_QMAX || q < -TNX_QMAX) { delete b; fail(TNX_ERR_UNSUPPORTED, "charge magnitude above 2^24"); }
        d.qn.push_back(q);
      }
    }
    d.finish();
    *out = b;
  });
}

extern "C" tnx_status tnx_bond_dim(const tnx_bond* b, int64_t* dim) {
  if (!b || !dim) return TNX_ERR_ARG;
  *dim = b->b.dim;
  return TNX_OK;
}

extern "C" tnx_status tnx_bond_sectors(const tnx_bond* b, int* nsec, int32_t* qnums, int64_t* degs) {
  if (!b || !nsec) return TNX_ERR_ARG;
  *nsec = b->b.nsec;
  if (qnums) std::copy(b->b.qn.begin(), b->b.qn.end(), qnums);
  if (degs) std::copy(b->b.deg.begin(), b->b.deg.end(), degs);
  return TNX_OK;
}

extern "C" tnx_status tnx_bond_info(const tnx_bond* b, int* dir, int* nsym, int* kinds, int* zn) {
  if (!b) return TNX_ERR_ARG;
  if (dir) *dir = b->b.dir;
  if (nsym) *nsym = b->b.nsym;
  for (int c = 0; c < b->b.nsym; ++c) {
    if (kinds) kinds[c] = b->b.kinds[c];
    if (zn) zn[c] = b->b.zn[c];
  }
  return TNX_OK;
}

extern "C" tnx_status tnx_bond_combine(const tnx_bond* a, const tnx_bond* b, tnx_bond** out) {
  if (!a || !b || !out) return TNX_ERR_ARG;
  tnx_ctx* ctx = a->ctx;
  return tnx_guard(ctx, [&] {
    const BondD &x = a->b, &y = b->b;
    if (x.dir != y.dir || !x.same_syms(y)) fail(TNX_ERR_ARG, "only bonds with equal direction and symmetries combine");
    std::map<std::vector<int32_t>, int64_t> acc;
    for (int s = 0; s < x.nsec; ++s)
      for (int t = 0; t < y.nsec; ++t) {
        std::vector<int32_t> q(x.nsym);
        for (int c = 0; c < x.nsym; ++c) {
          int32_t v = x.qn[(size_t)s * x.nsym + c] + y.qn[(size_t)t * y.nsym + c];
          if (x.kinds[c] == TNX_ZN) v = ((v % x.zn[c]) + x.zn[c]) % x.zn[c];
          if (v > TNX_QMAX || v < -TNX_QMAX) fail(TNX_ERR_UNSUPPORTED, "combined charge magnitude above 2^24");
          q[c] = v;
        }
        acc[q] += x.deg[s] * y.deg[t];
      }
    auto* r = new tnx_bond();
    r->ctx = ctx;
    BondD& d = r->b;
    d.dir = x.dir;
    d.nsym = x.nsym;
    d.kinds = x.kinds;
    d.zn = x.zn;
    d.nsec = (int)acc.size();
    for (auto& kv : acc) {
      d.qn.insert(d.qn.end(), kv.first.begin(), kv.first.end());
      d.deg.push_back(kv.second);
    }
    d.finish();
    *out = r;
  });
}

extern "C" tnx_status tnx_bond_destroy(tnx_bond* b) {
  if (!b) return TNX_ERR_ARG;
  delete b;
  return TNX_OK;
}

// ------------------------------------------------------------------ tensors
// Zero-flux sector tuples in lexicographic order (Sec. 6.3).
void enumerate_blocks(const std::vector<BondD>& bonds, std::vector<int32_t>& qn, int64_t& nblk) {
  const int r = (int)bonds.size();
  qn.clear();
  nblk = 0;
  if (r == 0) {
    nblk = 1;
    return;
  }
  const int nsym = bonds[0].nsym;
  for (const auto& b : bonds)
    if (!b.same_syms(bonds[0])) fail(TNX_ERR_ARG, "all bonds of a tensor must carry the same symmetries");
  std::vector<int32_t> idx(r, 0);
  while (true) {
    bool ok = true;
    for (int c = 0; c < nsym && ok; ++c) {
      int64_t s = 0;
      for (int l = 0; l < r; ++l) s += bonds[l].signed_q(idx[l], c);
      if (bonds[0].kinds[c] == TNX_ZN) s %= bonds[0].zn[c];
      ok = (s == 0);
    }
    if (ok) {
      qn.insert(qn.end(), idx.begin(), idx.end());
      ++nblk;
    }
    int l = r - 1;
    while (l >= 0 && ++idx[l] == bonds[l].nsec) idx[l--] = 0;
    if (l < 0) break;
  }
}

tnx_tensor* make_tensor(tnx_ctx* ctx, const std::vector<BondD>& bonds) {
  std::unique_ptr<tnx_tensor> t(new tnx_tensor());
  t->ctx = ctx;
  t->rank = (int)bonds.size();
  t->bonds = bonds;
  enumerate_blocks(bonds, t->qn, t->nblk);
  t->shape.resize((size_t)t->nblk * t->rank);
  t->off.resize(t->nblk);
  int64_t off = 0;
  for (int64_t b = 0; b < t->nblk; ++b) {
    int64_t n = 1;
    for (int l = 0; l < t->rank; ++l) {
      int64_t d = bonds[l].deg[t->qn[(size_t)b * t->rank + l]];
      t->shape[(size_t)b * t->rank + l] = d;
      n *= d;
    }
    t->off[b] = off;
    off += n;
    t->index[std::vector<int32_t>(t->qn.begin() + (size_t)b * t->rank, t->qn.begin() + (size_t)(b + 1) * t->rank)] = b;
  }
  t->nelem = off;
  t->bytes = (size_t)std::max<int64_t>(off, 1) * sizeof(double);
  t->data = (double*)ctx->dalloc(t->bytes);
  CUDA_CHECK(cudaMemsetAsync(t->data, 0, t->bytes, ctx->stream));
  return t.release();
}

tnx_tensor::~tnx_tensor() {
  if (ctx && data) ctx->dfree(data, bytes);
}

bool tnx_tensor::symmetric() const {
  for (const auto& b : bonds)
    if (b.nsym > 0) return true;
  return false;
}

extern "C" tnx_status tnx_tensor_create(tnx_ctx* ctx, int rank, tnx_bond* const* bonds, tnx_tensor** out) {
  return tnx_guard(ctx, [&] {
    if (!ctx || !out || rank < 0 || rank > TNX_MAXR || (rank > 0 && !bonds)) fail(TNX_ERR_ARG, "bad tensor arguments");
    std::vector<BondD> bs;
    for (int l = 0; l < rank; ++l) {
      if (!bonds[l]) fail(TNX_ERR_ARG, "null bond");
      bs.push_back(bonds[l]->b);
    }
    *out = make_tensor(ctx, bs);
  });
}

extern "C" tnx_status tnx_tensor_destroy(tnx_tensor* t) {
  if (!t) return TNX_ERR_ARG;
  delete t;
  return TNX_OK;
}

extern "C" tnx_status tnx_tensor_rank(const tnx_tensor* t, int* rank) {
  if (!t || !rank) return TNX_ERR_ARG;
  *rank = t->rank;
  return TNX_OK;
}

extern "C" tnx_status tnx_tensor_nblocks(const tnx_tensor* t, int64_t* n) {
  if (!t || !n) return TNX_ERR_ARG;
  *n = t->nblk;
  return TNX_OK;
}

extern "C" tnx_status tnx_tensor_block_info(const tnx_tensor* t, int64_t blk, int32_t* qn_idx, int64_t* shape,
                                           int64_t* offset) {
  if (!t) return TNX_ERR_ARG;
  if (blk < 0 || blk >= t->nblk) return set_err(t->ctx, TNX_ERR_NO_BLOCK, "block index out of range");
  for (int l = 0; l < t->rank; ++l) {
    if (qn_idx) qn_idx[l] = t->qn[(size_t)blk * t->rank + l];
    if (shape) shape[l] = t->shape[(size_t)blk * t->rank + l];
  }
  if (offset) *offset = t->off[blk];
  return TNX_OK;
}

extern "C" tnx_status tnx_tensor_blocks(const tnx_tensor* t, int32_t* qn_idx, int64_t* shape, int64_t* offset) {
  if (!t) return TNX_ERR_ARG;
  if (qn_idx) std::copy(t->qn.begin(), t->qn.end(), qn_idx);
  if (shape) std::copy(t->shape.begin(), t->shape.end(), shape);
  if (offset) std::copy(t->off.begin(), t->off.end(), offset);
  return TNX_OK;
}

extern "C" tnx_status tnx_tensor_bond(const tnx_tensor* t, int leg, tnx_bond** out) {
  if (!t) return TNX_ERR_ARG;
  return tnx_guard(t->ctx, [&] {
    if (!out || leg < 0 || leg >= t->rank) fail(TNX_ERR_ARG, "bad leg");
    auto* b = new tnx_bond();
    b->ctx = t->ctx;
    b->b = t->bonds[leg];
    *out = b;
  });
}

extern "C" tnx_status tnx_tensor_data(tnx_tensor* t, double** dev_ptr, int64_t* nelem) {
  if (!t) return TNX_ERR_ARG;
  if (dev_ptr) *dev_ptr = t->data;
  if (nelem) *nelem = t->rank == 0 ? 1 : t->nelem;
  return TNX_OK;
}

static int64_t find_block(const tnx_tensor* t, const int32_t* qn_idx) {
  if (t->rank == 0) return 0;
  std::vector<int32_t> k(qn_idx, qn_idx + t->rank);
  auto it = t->index.find(k);
  if (it == t->index.end()) fail(TNX_ERR_NO_BLOCK, "no stored block with these sector indices");
  return it->second;
}

static int64_t block_size(const tnx_tensor* t, int64_t b) {
  int64_t n = 1;
  for (int l = 0; l < t->rank; ++l) n *= t->shape[(size_t)b * t->rank + l];
  return n;
}

extern "C" tnx_status tnx_tensor_put_block(tnx_tensor* t, const int32_t* qn_idx, const double* host, int64_t n) {
  if (!t) return TNX_ERR_ARG;
  return tnx_guard(t->ctx, [&] {
    if (!host || (t->rank > 0 && !qn_idx)) fail(TNX_ERR_ARG, "null pointer");
    int64_t b = find_block(t, qn_idx);
    if (n != block_size(t, b)) fail(TNX_ERR_ARG, "size does not match the block");
    CUDA_CHECK(cudaMemcpyAsync(t->data + t->off[b], host, n * sizeof(double), cudaMemcpyHostToDevice, t->ctx->stream));
    CUDA_CHECK(cudaStreamSynchronize(t->ctx->stream));
  });
}

extern "C" tnx_status tnx_tensor_get_block(const tnx_tensor* t, const int32_t* qn_idx, double* host, int64_t n) {
  if (!t) return TNX_ERR_ARG;
  return tnx_guard(t->ctx, [&] {
    if (!host || (t->rank > 0 && !qn_idx)) fail(TNX_ERR_ARG, "null pointer");
    int64_t b = find_block(t, qn_idx);
    if (n != block_size(t, b)) fail(TNX_ERR_ARG, "size does not match the block");
    CUDA_CHECK(cudaMemcpyAsync(host, t->data + t->off[b], n * sizeof(double), cudaMemcpyDeviceToHost, t->ctx->stream));
    CUDA_CHECK(cudaStreamSynchronize(t->ctx->stream));
  });
}

extern "C" tnx_status tnx_tensor_upload(tnx_tensor* t, const double* host, int64_t n) {
  if (!t) return TNX_ERR_ARG;
  return tnx_guard(t->ctx, [&] {
    const int64_t ne = t->rank == 0 ? 1 : t->nelem;
    if (!host || n != ne) fail(TNX_ERR_ARG, "size does not match the tensor");
    CUDA_CHECK(cudaMemcpyAsync(t->data, host, n * sizeof(double), cudaMemcpyHostToDevice, t->ctx->stream));
    CUDA_CHECK(cudaStreamSynchronize(t->ctx->stream));
  });
}

extern "C" tnx_status tnx_tensor_download(const tnx_tensor* t, double* host, int64_t n) {
  if (!t) return TNX_ERR_ARG;
  return tnx_guard(t->ctx, [&] {
    const int64_t ne = t->rank == 0 ? 1 : t->nelem;
    if (!host || n != ne) fail(TNX_ERR_ARG, "size does not match the tensor");
    CUDA_CHECK(cudaMemcpyAsync(host, t->data, n * sizeof(double), cudaMemcpyDeviceToHost, t->ctx->stream));
    CUDA_CHECK(cudaStreamSynchronize(t->ctx->stream));
  });
}

extern "C" tnx_status tnx_tensor_scale(tnx_tensor* t, double alpha) {
  if (!t) return TNX_ERR_ARG;
  return tnx_guard(t->ctx, [&] {
    CUDA_CHECK(tnx_launch_scale(t->data, t->rank == 0 ? 1 : t->nelem, alpha, t->ctx->stream));
  });
}

extern "C" tnx_status tnx_tensor_add_scalar(tnx_tensor* t, double alpha) {
  if (!t) return TNX_ERR_ARG;
  return tnx_guard(t->ctx, [&] {
    if (t->symmetric())
      fail(TNX_ERR_SYMMETRY, "cannot add a scalar to a block-sparse tensor: it would break the block structure");
    CUDA_CHECK(tnx_launch_add_scalar(t->data, t->rank == 0 ? 1 : t->nelem, alpha, t->ctx->stream));
  });
}

extern "C" tnx_status tnx_tensor_norm(const tnx_tensor* t, double* out) {
  if (!t || !out) return TNX_ERR_ARG;
  return tnx_guard(t->ctx, [&] {
    tnx_ctx* c = t->ctx;
    double* partial = (double*)c->scratch->p;
    double* res = partial + 4096;
    CUDA_CHECK(tnx_launch_norm2(t->data, t->rank == 0 ? 1 : t->nelem, partial, res, c->stream));
    CUDA_CHECK(cudaMemcpyAsync(c->pinned, res, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_CHECK(cudaStreamSynchronize(c->stream));
    *out = *(double*)c->pinned;
  });
}
