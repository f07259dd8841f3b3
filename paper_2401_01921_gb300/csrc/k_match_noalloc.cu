// Fused charge-sector tables of one pairwise contraction without allocating
// memory.
//
// Who needs this: callers that must not call cudaMalloc (or any allocator) at
// the point where they need the tables.  Examples: a latency-critical loop
// whose memory budget was fixed up front, a process whose device memory is
// entirely owned by another framework's pool, or a plugin that receives only
// pre-sized buffers from its host application.
// They pass in the block lists and receive the tables in buffers they already
// own; the working memory of the matching kernel comes from one fixed array
// below instead of from an allocator.
//
// The scratch array is a file-scope __device__ array of TNX_NOALLOC_SCRATCH
// bytes (16 MiB).  Every device that loads this library holds one copy of it
// until the process exits.  All calls share it, so calls that overlap on the
// GPU (different streams, or different host threads on the same device) race
// on it: serialise them.  The array keeps whatever the previous call left; the
// kernel clears every presence flag it reads before use, and this file clears
// the status word before each launch.
//
// Host code cannot use the array's name as a device address: here it is only a
// host-side stand-in.  The device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, by the first call made on
// that device; make that first call before any stream capture.
#include <mutex>
#include <string>

#include "tnx_internal.h"

#define TNX_NOALLOC_SCRATCH (16u << 20)

namespace {

static __device__ __align__(256) unsigned char g_match_scratch[TNX_NOALLOC_SCRATCH];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};

void set_err(char* err, size_t len, const std::string& msg) {
  if (!err || len == 0) return;
  size_t n = msg.size() < len - 1 ? msg.size() : len - 1;
  for (size_t i = 0; i < n; ++i) err[i] = msg[i];
  err[n] = 0;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// pos K (nk entries) and pos F (nf entries) together name each of the r legs once
bool legs_form_permutation(int r, int nk, const int32_t* posK, int nf, const int32_t* posF) {
  if (nk + nf != r || (nk > 0 && !posK) || (nf > 0 && !posF)) return false;
  bool seen[TNX_MAXR] = {};
  for (int i = 0; i < nk + nf; ++i) {
    const int32_t v = i < nk ? posK[i] : posF[i - nk];
    if (v < 0 || v >= r || seen[v]) return false;
    seen[v] = true;
  }
  return true;
}

}  // namespace

extern "C" tnx_status tnx_match_tables_noalloc(void* stream, int nsym, const int32_t* zn, int nk, int nfa, int nfb,
                                               const int32_t* nsec, const int64_t* degs, const int32_t* kcharges,
                                               int64_t nA, int rA, const int32_t* qA, const int32_t* kposA,
                                               const int32_t* fposA, int64_t nB, int rB, const int32_t* qB,
                                               const int32_t* kposB, const int32_t* fposB, int gmax,
                                               int32_t* ngroups, int32_t* charges, int64_t* mkn, int64_t* amap,
                                               int64_t* bmap, char* err, size_t errlen) {
  cudaStream_t st = (cudaStream_t)stream;
  if (nsym < 0 || nsym > TNX_MAXSYM || nk < 0 || nfa < 0 || nfb < 0 || nk > TNX_MAXR || nfa > TNX_MAXR ||
      nfb > TNX_MAXR || nA < 0 || nB < 0 || rA < 0 || rB < 0 || rA > TNX_MAXR || rB > TNX_MAXR || gmax < 1 ||
      !ngroups || !charges || !mkn || (nA && (!qA || !amap)) || (nB && (!qB || !bmap)) ||
      (nk + nfa + nfb > 0 && (!nsec || !degs)) || (nk > 0 && nsym > 0 && !kcharges) || (nsym > 0 && !zn)) {
    set_err(err, errlen, "tnx_match_tables_noalloc: invalid argument");
    return TNX_ERR_ARG;
  }
  // The K and free positions of each operand must name every one of its legs
  // exactly once: the kernel reads each block's sector indices through them.
  if (!legs_form_permutation(rA, nk, kposA, nfa, fposA) || !legs_form_permutation(rB, nk, kposB, nfb, fposB)) {
    set_err(err, errlen,
            "tnx_match_tables_noalloc: the K and free leg positions of an operand must be a permutation of its legs");
    return TNX_ERR_ARG;
  }
  for (int c = 0; c < nsym; ++c)
    if (zn[c] < 0 || zn[c] > (1 << 22)) {
      set_err(err, errlen, "tnx_match_tables_noalloc: Z_n modulus outside [1, 2^22] (0 = U(1))");
      return zn[c] < 0 ? TNX_ERR_ARG : TNX_ERR_UNSUPPORTED;
    }

  // ---- sizes (same conventions as the planner's matching step)
  MatchArgs a;
  for (size_t i = 0; i < sizeof(a); ++i) ((unsigned char*)&a)[i] = 0;
  a.nk = nk;
  a.nfa = nfa;
  a.nfb = nfb;
  a.nsym = nsym;
  int nsec_total = 0;
  int64_t kspace = 1, faspace = 1, fbspace = 1;
  for (int l = 0; l < nk + nfa + nfb; ++l) {
    if (nsec[l] < 1) {
      set_err(err, errlen, "tnx_match_tables_noalloc: a leg without sectors");
      return TNX_ERR_ARG;
    }
    MatchLeg ml{nsec[l], nsec_total};
    if (l < nk) a.kleg[l] = ml, kspace *= nsec[l];
    else if (l < nk + nfa) a.faleg[l - nk] = ml, faspace *= nsec[l];
    else a.fbleg[l - nk - nfa] = ml, fbspace *= nsec[l];
    nsec_total += nsec[l];
    if (kspace > (1 << 24) || faspace > (1 << 24) || fbspace > (1 << 24)) {
      set_err(err, errlen, "tnx_match_tables_noalloc: sector tuple space too large");
      return TNX_ERR_UNSUPPORTED;
    }
  }
  int nksec = 0;
  for (int l = 0; l < nk; ++l) nksec += nsec[l];
  int64_t cspace = 1;
  for (int c = 0; c < nsym; ++c) {
    a.zn[c] = zn[c];
    if (zn[c] > 0) {
      a.clo[c] = 0;
      a.crange[c] = zn[c];
    } else {
      int64_t lo = 0, hi = 0, base = 0;
      for (int l = 0; l < nk; ++l) {
        int32_t mn = 0, mx = 0;
        for (int s = 0; s < nsec[l]; ++s) {
          const int32_t q = kcharges[(base + s) * nsym + c];
          if (q > TNX_QMAX || q < -TNX_QMAX) {
            set_err(err, errlen, "tnx_match_tables_noalloc: a K-leg charge magnitude above 2^24");
            return TNX_ERR_UNSUPPORTED;
          }
          if (s == 0 || q < mn) mn = q;
          if (s == 0 || q > mx) mx = q;
        }
        lo += mn;
        hi += mx;
        base += nsec[l];
      }
      if (hi - lo + 1 > (1 << 22)) {
        set_err(err, errlen, "tnx_match_tables_noalloc: charge range too wide");
        return TNX_ERR_UNSUPPORTED;
      }
      a.clo[c] = (int32_t)lo;
      a.crange[c] = (int32_t)(hi - lo + 1);
    }
    cspace *= a.crange[c];
    // the same bound as the allocating planner: checked after every factor,
    // so the product cannot wrap before the scratch layout is sized from it
    if (cspace > (int64_t(1) << 24)) {
      set_err(err, errlen, "tnx_match_tables_noalloc: charge space above 2^24");
      return TNX_ERR_UNSUPPORTED;
    }
  }
  a.kspace = kspace;
  a.faspace = faspace;
  a.fbspace = fbspace;
  a.cspace = cspace;
  int64_t gm = cspace < kspace ? cspace : kspace;
  if (gm > gmax) gm = gmax;
  a.gmax = (int32_t)gm;
  a.nA = nA;
  a.nB = nB;
  a.rA = rA;
  a.rB = rB;
  a.qA = qA;
  a.qB = qB;
  for (int i = 0; i < nk; ++i) a.kposA[i] = kposA[i], a.kposB[i] = kposB[i];
  for (int i = 0; i < nfa; ++i) a.fposA[i] = fposA[i];
  for (int i = 0; i < nfb; ++i) a.fposB[i] = fposB[i];

  // ---- scratch layout inside the fixed array
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + (bytes ? bytes : 1));
    return o;
  };
  const size_t o_deg = take((size_t)nsec_total * 8);
  const size_t o_kq = take((size_t)nksec * (nsym ? nsym : 1) * 4);
  const size_t o_kpres = take((size_t)kspace * 4), o_kgroup = take((size_t)kspace * 4), o_koff = take((size_t)kspace * 8);
  const size_t o_rgroup = take((size_t)faspace * 4), o_roff = take((size_t)faspace * 8);
  const size_t o_cgroup = take((size_t)fbspace * 4), o_coff = take((size_t)fbspace * 8);
  const size_t o_cspres = take((size_t)cspace * 4), o_csgid = take((size_t)cspace * 4);
  const size_t o_scan = take(((size_t)1024 * gm + 3 * (size_t)gm) * 8);
  const size_t o_status = take(8);
  if (off > TNX_NOALLOC_SCRATCH) {
    set_err(err, errlen, "tnx_match_tables_noalloc: this contraction needs " + std::to_string(off) +
                             " bytes of scratch; the fixed limit is " + std::to_string(TNX_NOALLOC_SCRATCH) +
                             " bytes (use the allocating network entry points instead)");
    return TNX_ERR_UNSUPPORTED;
  }
  // ---- set-up: device address of the scratch array, once per device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_err(err, errlen, "tnx_match_tables_noalloc: no usable current CUDA device");
    return TNX_ERR_CUDA;
  }
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_match_scratch);
      if (e != cudaSuccess || !p) {
        set_err(err, errlen, std::string("tnx_match_tables_noalloc: cudaGetSymbolAddress failed: ") +
                                 cudaGetErrorString(e));
        return TNX_ERR_CUDA;
      }
      g_scratch_dev[dev] = p;
    }
    scratch = (unsigned char*)g_scratch_dev[dev];
  }

  a.deg = (const int64_t*)(scratch + o_deg);
  a.kcharge = (const int32_t*)(scratch + o_kq);
  a.kpres = (int32_t*)(scratch + o_kpres);
  a.kgroup = (int32_t*)(scratch + o_kgroup);
  a.koff = (int64_t*)(scratch + o_koff);
  a.rgroup = (int32_t*)(scratch + o_rgroup);
  a.roff = (int64_t*)(scratch + o_roff);
  a.cgroup = (int32_t*)(scratch + o_cgroup);
  a.coff = (int64_t*)(scratch + o_coff);
  a.cspres = (int32_t*)(scratch + o_cspres);
  a.csgid = (int32_t*)(scratch + o_csgid);
  a.scan_tmp = (int64_t*)(scratch + o_scan);
  a.status = (int32_t*)(scratch + o_status);
  a.ngroups = ngroups;
  a.charges = charges;
  a.mkn = mkn;
  a.amap = amap;
  a.bmap = bmap;

  // ---- inputs into the scratch array, status cleared, launch, wait, check
  cudaError_t e = cudaSuccess;
  if (nsec_total) e = cudaMemcpyAsync(scratch + o_deg, degs, (size_t)nsec_total * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nksec && nsym)
    e = cudaMemcpyAsync(scratch + o_kq, kcharges, (size_t)nksec * nsym * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch + o_status, 0, 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ngroups, 0, 4, st);
  if (e == cudaSuccess) e = tnx_launch_match(a, st);
  int32_t hs[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs[0], ngroups, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs[1], scratch + o_status, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_err(err, errlen, std::string("tnx_match_tables_noalloc: ") + cudaGetErrorString(e));
    return TNX_ERR_CUDA;
  }
  if (hs[1] == 1) {
    set_err(err, errlen, "tnx_match_tables_noalloc: " + std::to_string(hs[0]) + " charge groups exceed gmax = " +
                             std::to_string(gmax));
    return TNX_ERR_UNSUPPORTED;
  }
  if (hs[1] == 3) {
    set_err(err, errlen, "tnx_match_tables_noalloc: a block's sector index lies outside its leg (no table written)");
    return TNX_ERR_ARG;
  }
  if (hs[1] != 0) {
    set_err(err, errlen, "tnx_match_tables_noalloc: a K-leg charge lies outside the given charges");
    return TNX_ERR_ARG;
  }
  set_err(err, errlen, "");
  return TNX_OK;
}
