// Host-only internal declarations (C++).
#pragma once

#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "tnx_internal.h"

struct TnxError {
  int code;
  std::string msg;
};

[[noreturn]] inline void fail(int code, const std::string& msg) { throw TnxError{code, msg}; }

#define CUDA_CHECK(x)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (x);                                                                    \
    if (e_ != cudaSuccess) fail(TNX_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct DevBuf;

struct ProfRec {
  cudaEvent_t a, b;
  int cls;
  double work;
};

struct tnx_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  tnx_alloc_fn alloc = nullptr;
  tnx_free_fn fre = nullptr;
  void* user = nullptr;
  std::string err;
  DevBuf* scratch = nullptr;   // small device scratch (norm partials)
  void* pinned = nullptr;      // small pinned host buffer
  int32_t* d_status = nullptr; // device status word written by bounded waits (0 = ok)
  bool use_graphs = true;      // capture applies / Lanczos solves in CUDA graphs (needs a non-default stream)
  // profiler (CUDA events around kernel classes)
  uint32_t prof = 0;                 // bit c set: kernel class c is timed
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> event_pool;
  double prof_ms[TNX_KC_COUNT] = {};
  int64_t prof_n[TNX_KC_COUNT] = {};
  double prof_work[TNX_KC_COUNT] = {};
  std::vector<ProfRec>* capture_recs = nullptr;   // set while a graph is being captured
  cudaEvent_t get_event();
  void* dalloc(size_t n);
  void dfree(void* p, size_t n);
};

// Brackets the launches made in its scope with two events when profiling is on.
struct ProfScope {
  tnx_ctx* c;
  cudaStream_t st;
  int cls;
  double work;
  cudaEvent_t a = nullptr;
  ProfScope(tnx_ctx* c_, cudaStream_t s_, int cls_, double work_);
  ~ProfScope();
};

struct DevBuf {
  tnx_ctx* ctx = nullptr;
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf(tnx_ctx* c, size_t n);
  ~DevBuf();
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

struct BondD {
  int dir = 0;
  int nsym = 0;
  std::vector<int> kinds, zn;
  int nsec = 0;
  std::vector<int32_t> qn;   // nsec * nsym
  std::vector<int64_t> deg;  // nsec
  std::vector<int64_t> off;  // nsec + 1
  int64_t dim = 0;
  int32_t signed_q(int s, int c) const;   // charge as it enters the flux
  bool same_syms(const BondD& o) const;
  bool operator==(const BondD& o) const;
  bool operator!=(const BondD& o) const { return !(*this == o); }
  void finish();
  std::string key() const;
};

struct tnx_bond {
  tnx_ctx* ctx = nullptr;
  BondD b;
};

struct tnx_tensor {
  tnx_ctx* ctx = nullptr;
  int rank = 0;
  std::vector<BondD> bonds;
  int64_t nblk = 0;
  std::vector<int32_t> qn;      // nblk * rank
  std::vector<int64_t> shape;   // nblk * rank
  std::vector<int64_t> off;     // nblk
  int64_t nelem = 0;
  double* data = nullptr;
  size_t bytes = 0;
  std::map<std::vector<int32_t>, int64_t> index;
  ~tnx_tensor();
  bool symmetric() const;
};

tnx_status tnx_guard(tnx_ctx* ctx, const std::function<void()>& f);
// add the timings of events recorded inside a graph (after the graph ran)
void prof_accumulate(tnx_ctx* ctx, const std::vector<ProfRec>& recs);
// after a stream sync: fail with TNX_ERR_TIMEOUT if a device wait ran out (and clear it)
void check_device_status(tnx_ctx* ctx);
void check_contractible(const BondD& a, const BondD& b, const std::string& label);
void enumerate_blocks(const std::vector<BondD>& bonds, std::vector<int32_t>& qn, int64_t& nblk);
tnx_tensor* make_tensor(tnx_ctx* ctx, const std::vector<BondD>& bonds);
