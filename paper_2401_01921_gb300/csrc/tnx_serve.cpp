// Serving loop with continuous batching (no counterpart in the paper).
//
// Requests are H_eff*psi applies or Lanczos solves on networks whose
// environment tensors stay resident on the device.  A worker thread admits
// requests from the queue whenever (a) one of the server's stream slots is
// free, (b) the request's network is not already running another request, and
// (c) the bytes its network will hold while it runs (plan buffers, sized
// before anything is allocated, plus the Lanczos workspace) fit the HBM
// budget next to the bytes already resident - idle resident networks are
// evicted least recently used first to make room; a request that could not
// fit even alone fails with TNX_ERR_OOM.  Sizing and planning run with the
// server's lock released.  Admitted requests run on their own CUDA streams, so
// the work of requests that arrive while others are on the GPU overlaps on the
// device; completions are detected with CUDA events and reported to waiters.
// Latency = completion seen by the worker - submission (host steady clock).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "tnx_plan.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  tnx_network* net = nullptr;
  int slot = -1;
  tnx_tensor* vec = nullptr;
  tnx_tensor* out = nullptr;
  int kind = 0;        // TNX_REQ_APPLY / TNX_REQ_LANCZOS
  int nsteps = 0;
  Clock::time_point submitted, started, finished;
  int status = 1;      // 1 = pending/running, 0 = done, < 0 = error code
  std::string err;
  double eval = 0.0;
  int matvecs = 0;
  int stream_slot = -1;
  size_t need = 0;     // resident bytes of its network while it runs (0 = not sized yet)
  cudaEvent_t done = nullptr;
};

}  // namespace

struct tnx_server {
  tnx_ctx* ctx = nullptr;
  int max_slots = 0;
  size_t budget = 0;
  std::vector<cudaStream_t> streams;
  std::vector<int64_t> slot_req;          // request id per stream slot, -1 free
  double* pinned = nullptr;               // 2 doubles of results per slot
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, Request> reqs;
  std::unordered_map<tnx_network*, int64_t> busy;     // network -> running request
  std::list<tnx_network*> lru;                        // resident networks, most recent at the back
  size_t used = 0;
  std::unordered_map<tnx_network*, size_t> resident;  // bytes counted per resident network
  int64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  // stats
  int64_t completed = 0, evictions = 0;
  size_t peak_used = 0;
};

namespace {

void touch(tnx_server* S, tnx_network* net) {
  S->lru.remove(net);
  S->lru.push_back(net);
}

void account(tnx_server* S, tnx_network* net) {
  const size_t b = tnx_network_resident_bytes(net);
  S->used -= S->resident[net];
  S->resident[net] = b;
  S->used += b;
  S->peak_used = std::max(S->peak_used, S->used);
}

// Make room for `need` more bytes by evicting idle networks (LRU); true if it fits.
// An evicted network keeps no plan or workspace; its next request is sized
// (and planned) again.
bool make_room(tnx_server* S, size_t need, tnx_network* keep) {
  while (S->used + need > S->budget) {
    tnx_network* victim = nullptr;
    for (tnx_network* n : S->lru)
      if (n != keep && !S->busy.count(n) && S->resident[n] > 0) {
        victim = n;
        break;
      }
    if (!victim) return false;
    tnx_network_evict(victim);
    S->used -= S->resident[victim];
    S->resident[victim] = 0;
    S->lru.remove(victim);
    S->evictions++;
  }
  return true;
}

// Runs f and turns a failure into (status, message) without touching the
// context's error string (the caller's thread owns it).
template <class F>
int run_caught(F&& f, std::string& err) {
  try {
    f();
    return TNX_OK;
  } catch (const TnxError& e) {
    err = e.msg;
    return e.code;
  } catch (const std::exception& e) {
    err = e.what();
    return TNX_ERR_ARG;
  }
}

void bind_vector(Request& r) {
  NetTensor& nt = r.net->ts[r.slot];
  nt.t = r.vec;
  nt.perm.assign(r.vec->rank, 0);
  for (int j = 0; j < r.vec->rank; ++j) nt.perm[j] = j;
}

// Device bytes the request's network holds while the request runs: its plan
// (sized without allocating when it is not resident) and its Lanczos
// workspace (a solve allocates one for its step count; an apply keeps
// whatever the network holds).  Worker thread, lock released, network marked
// busy.
size_t request_bytes(Request& r) {
  bind_vector(r);
  const size_t plan = tnx_network_plan_bytes(r.net);
  const size_t lz = r.kind == TNX_REQ_LANCZOS ? tnx_lanczos_workspace_bytes(r.vec->nelem, r.nsteps)
                                              : tnx_network_lanczos_bytes(r.net);
  return plan + lz;
}

void finish_failed(tnx_server* S, Request& r, int code, const std::string& err) {
  r.status = code;
  r.err = err;
  r.finished = Clock::now();
  S->cv_done.notify_all();
}

// Enqueue request r on stream slot k (worker thread, lock released; the
// network is marked busy and the slot taken).  Builds the plan if needed.
int start(tnx_server* S, Request& r, int k, std::string& err) {
  cudaStream_t st = S->streams[k];
  return run_caught([&] {
    bind_vector(r);
    if (r.kind == TNX_REQ_APPLY) tnx_apply_enqueue(r.net, r.out, st);
    else tnx_lanczos_enqueue(r.net, r.slot, r.vec, r.nsteps, r.out, st, S->pinned + 2 * k);
    CUDA_CHECK(cudaEventRecord(r.done, st));
  }, err);
}

void worker_loop(tnx_server* S) {
  cudaSetDevice(S->ctx->device);
  std::unique_lock<std::mutex> lock(S->mu);
  while (!S->stop) {
    bool progress = false;
    // completions
    for (int k = 0; k < S->max_slots; ++k) {
      const int64_t id = S->slot_req[k];
      if (id < 0) continue;
      Request& r = S->reqs[id];
      const cudaError_t q = cudaEventQuery(r.done);
      if (q == cudaErrorNotReady) continue;
      r.finished = Clock::now();
      if (q != cudaSuccess) {
        cudaGetLastError();
        r.status = TNX_ERR_CUDA;
        r.err = cudaGetErrorString(q);
      } else {
        r.status = 0;
        if (r.kind == TNX_REQ_LANCZOS) {
          r.eval = S->pinned[2 * k];
          r.matvecs = ((int32_t*)(S->pinned + 2 * k + 1))[0];
        }
      }
      S->busy.erase(r.net);
      S->slot_req[k] = -1;
      S->completed++;
      progress = true;
      S->cv_done.notify_all();
    }
    // admissions, first fit in arrival order.  Sizing and starting release
    // the lock (planning runs kernels and waits for them); the scan restarts
    // afterwards because submissions may have changed the queue meanwhile.
    bool rescan = true;
    while (rescan && !S->stop) {
      rescan = false;
      for (auto it = S->queue.begin(); it != S->queue.end();) {
        int k = -1;
        for (int q = 0; q < S->max_slots; ++q)
          if (S->slot_req[q] < 0) { k = q; break; }
        if (k < 0) break;
        const int64_t id = *it;
        Request& r = S->reqs[id];
        if (S->busy.count(r.net)) { ++it; continue; }
        if (r.need == 0) {
          // size it: the network is marked busy so nothing else touches it
          S->busy[r.net] = id;
          lock.unlock();
          std::string err;
          size_t need = 0;
          const int code = run_caught([&] { need = request_bytes(r); }, err);
          lock.lock();
          S->busy.erase(r.net);
          if (code != TNX_OK) {
            S->queue.erase(std::find(S->queue.begin(), S->queue.end(), id));
            finish_failed(S, r, code, err);
          } else {
            r.need = std::max<size_t>(need, 1);
          }
          progress = rescan = true;
          break;
        }
        if (r.need > S->budget) {
          it = S->queue.erase(it);
          finish_failed(S, r, TNX_ERR_OOM,
                        "the request needs " + std::to_string(r.need) + " resident bytes, above the server's budget of " +
                            std::to_string(S->budget));
          progress = true;
          continue;
        }
        const size_t have = S->resident[r.net];
        const size_t extra = r.need > have ? r.need - have : 0;
        if (!make_room(S, extra, r.net)) { ++it; continue; }
        // admitted: reserve its bytes, take the slot, enqueue without the lock
        S->used += extra;
        S->resident[r.net] = have + extra;
        S->peak_used = std::max(S->peak_used, S->used);
        S->busy[r.net] = id;
        S->slot_req[k] = id;
        r.stream_slot = k;
        r.started = Clock::now();
        touch(S, r.net);
        S->queue.erase(it);
        lock.unlock();
        std::string err;
        const int code = start(S, r, k, err);
        lock.lock();
        account(S, r.net);
        if (code != TNX_OK) {
          S->busy.erase(r.net);
          S->slot_req[k] = -1;
          finish_failed(S, r, code, err);
        }
        progress = rescan = true;
        break;
      }
    }
    if (!progress) S->cv_work.wait_for(lock, std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" tnx_status tnx_server_create(tnx_ctx* ctx, int max_slots, size_t hbm_budget_bytes, tnx_server** out) {
  return tnx_guard(ctx, [&] {
    if (!ctx || !out || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0) fail(TNX_ERR_ARG, "bad server arguments");
    std::unique_ptr<tnx_server> S(new tnx_server());
    S->ctx = ctx;
    S->max_slots = max_slots;
    S->budget = hbm_budget_bytes;
    for (int k = 0; k < max_slots; ++k) {
      cudaStream_t st;
      CUDA_CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      S->streams.push_back(st);
    }
    S->slot_req.assign(max_slots, -1);
    CUDA_CHECK(cudaMallocHost(&S->pinned, sizeof(double) * 2 * max_slots));
    tnx_server* raw = S.get();
    S->worker = std::thread(worker_loop, raw);
    *out = S.release();
  });
}

extern "C" tnx_status tnx_server_destroy(tnx_server* S) {
  if (!S) return TNX_ERR_ARG;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto st : S->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (auto& kv : S->reqs)
    if (kv.second.done) cudaEventDestroy(kv.second.done);
  if (S->pinned) cudaFreeHost(S->pinned);
  delete S;
  return TNX_OK;
}

extern "C" tnx_status tnx_server_submit(tnx_server* S, tnx_network* net, const char* vec_slot, tnx_tensor* vec, int kind,
                                        int nsteps, tnx_tensor* out, int64_t* id) {
  if (!S) return TNX_ERR_ARG;
  return tnx_guard(S->ctx, [&] {
    if (!net || !vec_slot || !vec || !id || net->ctx != S->ctx) fail(TNX_ERR_ARG, "bad request");
    if (kind != TNX_REQ_APPLY && kind != TNX_REQ_LANCZOS) fail(TNX_ERR_ARG, "unknown request kind");
    if (kind == TNX_REQ_APPLY && !out) fail(TNX_ERR_ARG, "an apply needs an output tensor");
    if (kind == TNX_REQ_LANCZOS && (nsteps < 1 || nsteps > 500)) fail(TNX_ERR_ARG, "bad Lanczos step count");
    const int slot = tnx_network_slot(net, vec_slot);
    if (slot < 0) fail(TNX_ERR_NETWORK, std::string("no tensor named '") + vec_slot + "'");
    Request r;
    r.net = net;
    r.slot = slot;
    r.vec = vec;
    r.out = out;
    r.kind = kind;
    r.nsteps = nsteps;
    r.submitted = Clock::now();
    CUDA_CHECK(cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming));
    {
      std::lock_guard<std::mutex> lock(S->mu);
      r.id = S->next_id++;
      *id = r.id;
      S->reqs[r.id] = r;
      S->queue.push_back(r.id);
    }
    S->cv_work.notify_all();
  });
}

extern "C" tnx_status tnx_server_wait(tnx_server* S, int64_t id, int timeout_ms, double* eval, int* matvecs,
                                      double* latency_ms) {
  if (!S) return TNX_ERR_ARG;
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) {
    S->ctx->err = "unknown request id";
    return TNX_ERR_ARG;
  }
  auto pred = [&] { return S->reqs[id].status <= 0; };
  if (timeout_ms < 0) S->cv_done.wait(lock, pred);
  else if (!S->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), pred)) return TNX_ERR_TIMEOUT;
  Request& r = S->reqs[id];
  if (eval) *eval = r.eval;
  if (matvecs) *matvecs = r.matvecs;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r.finished - r.submitted).count();
  const int st = r.status;
  if (st < 0) S->ctx->err = r.err;
  cudaEventDestroy(r.done);
  S->reqs.erase(id);
  return st < 0 ? st : TNX_OK;
}

extern "C" tnx_status tnx_server_stats(tnx_server* S, int64_t* completed, int64_t* evictions, size_t* used_bytes,
                                       size_t* peak_bytes) {
  if (!S) return TNX_ERR_ARG;
  std::lock_guard<std::mutex> lock(S->mu);
  if (completed) *completed = S->completed;
  if (evictions) *evictions = S->evictions;
  if (used_bytes) *used_bytes = S->used;
  if (peak_bytes) *peak_bytes = S->peak_used;
  return TNX_OK;
}
