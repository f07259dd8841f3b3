// Two-site DMRG sweep (Sec. 11 of arXiv 2401.01921: the benchmark around Fig.
// "Hpsi_fig"; the paper's own sweep is an example in its user guide), built
// from the library's calls: the two-site wavefunction A_i A_{i+1} and the
// environment updates L.A.W.A^dagger / A.W.R.A^dagger are network launches,
// the lowest eigenvector of H_eff = (L, W, W, R) is a Lanczos solve on the
// H_eff network, and the split is the block-sparse SVD with truncation.
//
// Conventions (the H_eff ones): A_i[a IN, s IN, b OUT], L[a OUT, w OUT, a' IN],
// R[b IN, w IN, b' OUT], W[wL IN, s' IN, s OUT, wR OUT].  L[i] holds sites
// 0..i-1, R[i] sites i..N-1; L[0] and R[N] are one-dimensional edges that
// select the MPO's left row / right column.  A sweep runs the bond (i, i+1)
// from left to right (A_i = U, A_{i+1} = S V^dagger, then L[i+1]) and back
// (A_{i+1} = V^dagger, A_i = U S, then R[i+1]).
#include <chrono>

#include "tnx_plan.h"

void tnx_svd_run(tnx_tensor* t, int rowrank, int64_t keepdim, double err, const int64_t* min_blockdim, int nmin,
                 int absorb, tnx_tensor** U_out, tnx_tensor** S_out, tnx_tensor** V_out, double* trunc_err,
                 double* discarded, int* sweeps_out);

namespace {

const char* TWO_SITE = "A1: a, s1, m\nA2: m, s2, b\nTOUT: a, s1, s2, b\n";
const char* HEFF = "L: a, w0, ap\npsi: a, s1, s2, b\nW1: w0, s1p, s1, w1\nW2: w1, s2p, s2, w2\nR: b, w2, bp\n"
                   "TOUT: ap, s1p, s2p, bp\n";
const char* ENV_L = "L: a, w, ap\nA: a, s, b\nW: w, sp, s, wp\nAd: ap, sp, bp\nTOUT: b, wp, bp\n";
const char* ENV_R = "A: a, s, b\nW: w, sp, s, wp\nR: b, wp, bp\nAd: ap, sp, bp\nTOUT: a, w, ap\n";

using TPtr = std::unique_ptr<tnx_tensor>;

struct NetDel {
  void operator()(tnx_network* n) const { tnx_network_destroy(n); }
};
using NPtr = std::unique_ptr<tnx_network, NetDel>;

void chk(tnx_ctx* c, tnx_status s) {
  if (s != TNX_OK) fail(s, c->err);
}

BondD edge_bond(const BondD& like, int dir, const std::vector<int32_t>& q) {
  BondD b;
  b.nsym = like.nsym;
  b.kinds = like.kinds;
  b.zn = like.zn;
  b.dir = like.nsym ? dir : TNX_BD_REG;
  b.nsec = 1;
  b.qn = q;
  b.deg = {1};
  b.finish();
  return b;
}

BondD redirected(BondD b, int dir) {
  b.dir = b.nsym ? dir : TNX_BD_REG;
  return b;
}

// (sector, offset inside it) of dense index x of bond b
std::pair<int, int64_t> locate(const BondD& b, int64_t x) {
  for (int k = 0; k < b.nsec; ++k)
    if (x >= b.off[k] && x < b.off[k + 1]) return {k, x - b.off[k]};
  fail(TNX_ERR_ARG, "index outside the bond");
}

void set_one(tnx_tensor* t, const std::vector<int32_t>& qn, int64_t elem) {
  auto it = t->index.find(qn);
  if (it == t->index.end()) fail(TNX_ERR_ARG, "the edge or product-state entry breaks the charge rule");
  const double one = 1.0;
  CUDA_CHECK(cudaMemcpyAsync(t->data + t->off[it->second] + elem, &one, sizeof(double), cudaMemcpyHostToDevice,
                             t->ctx->stream));
  CUDA_CHECK(cudaStreamSynchronize(t->ctx->stream));
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct tnx_dmrg {
  tnx_ctx* ctx = nullptr;
  int N = 0;
  TPtr W;
  std::vector<TPtr> A, L, R;
  NPtr two, heff, envl, envr;
};

namespace {

tnx_tensor* launch(tnx_network* net, const std::vector<std::pair<const char*, tnx_tensor*>>& ins) {
  tnx_ctx* c = net->ctx;
  for (auto& kv : ins) chk(c, tnx_network_put(net, kv.first, kv.second, 0, nullptr));
  tnx_tensor* out = nullptr;
  chk(c, tnx_network_launch(net, &out));
  return out;
}

void env_left(tnx_dmrg* d, int i) {   // L[i+1] from L[i] and A_i
  tnx_tensor* ad = nullptr;
  chk(d->ctx, tnx_tensor_dagger(d->A[i].get(), &ad));
  TPtr Ad(ad);
  d->L[i + 1].reset(launch(d->envl.get(), {{"L", d->L[i].get()}, {"A", d->A[i].get()}, {"W", d->W.get()},
                                           {"Ad", Ad.get()}}));
  chk(d->ctx, tnx_sync(d->ctx));
}

void env_right(tnx_dmrg* d, int i) {  // R[i] from A_i and R[i+1]
  tnx_tensor* ad = nullptr;
  chk(d->ctx, tnx_tensor_dagger(d->A[i].get(), &ad));
  TPtr Ad(ad);
  d->R[i].reset(launch(d->envr.get(), {{"A", d->A[i].get()}, {"W", d->W.get()}, {"R", d->R[i + 1].get()},
                                       {"Ad", Ad.get()}}));
  chk(d->ctx, tnx_sync(d->ctx));
}

}  // namespace

extern "C" tnx_status tnx_dmrg_create(tnx_ctx* ctx, int nsites, const tnx_tensor* W, int left_w, int right_w,
                                      const int32_t* states, tnx_dmrg** out) {
  return tnx_guard(ctx, [&] {
    if (!ctx || !W || !states || !out || nsites < 2) fail(TNX_ERR_ARG, "bad DMRG arguments");
    if (W->rank != 4) fail(TNX_ERR_ARG, "the MPO tensor has legs [wL, s', s, wR]");
    const BondD &wl = W->bonds[0], &sp = W->bonds[1], &sn = W->bonds[2], &wr = W->bonds[3];
    if (wl.nsym && (wl.dir != TNX_BD_IN || sp.dir != TNX_BD_IN || sn.dir != TNX_BD_OUT || wr.dir != TNX_BD_OUT))
      fail(TNX_ERR_BOND_MISMATCH, "MPO legs must be [wL IN, s' IN, s OUT, wR OUT]");
    if (left_w < 0 || left_w >= wl.dim || right_w < 0 || right_w >= wr.dim) fail(TNX_ERR_ARG, "edge channel");
    std::unique_ptr<tnx_dmrg> d(new tnx_dmrg());
    d->ctx = ctx;
    d->N = nsites;
    tnx_tensor* w = nullptr;
    // an owned copy of W: the dagger of its dagger
    {
      tnx_tensor* wd = nullptr;
      chk(ctx, tnx_tensor_dagger(W, &wd));
      TPtr tmp(wd);
      chk(ctx, tnx_tensor_dagger(wd, &w));
    }
    d->W.reset(w);
    const int nsym = wl.nsym;
    std::vector<int32_t> q(nsym, 0);
    const BondD phys = redirected(sp, TNX_BD_IN);
    for (int i = 0; i < nsites; ++i) {
      if (states[i] < 0 || states[i] >= phys.dim) fail(TNX_ERR_ARG, "product state outside the physical bond");
      const auto loc = locate(phys, states[i]);
      std::vector<int32_t> q2 = q;
      for (int c = 0; c < nsym; ++c) {
        q2[c] += phys.signed_q(loc.first, c);
        if (phys.kinds[c] == TNX_ZN) q2[c] = ((q2[c] % phys.zn[c]) + phys.zn[c]) % phys.zn[c];
      }
      TPtr a(make_tensor(ctx, {edge_bond(wl, TNX_BD_IN, q), phys, edge_bond(wl, TNX_BD_OUT, q2)}));
      set_one(a.get(), {0, loc.first, 0}, loc.second);
      d->A.push_back(std::move(a));
      q = q2;
    }
    const std::vector<int32_t> zero(nsym, 0);
    d->L.resize(nsites + 1);
    d->R.resize(nsites + 1);
    d->L[0].reset(make_tensor(ctx, {edge_bond(wl, TNX_BD_OUT, zero), redirected(wl, TNX_BD_OUT),
                                    edge_bond(wl, TNX_BD_IN, zero)}));
    const auto lw = locate(wl, left_w);
    set_one(d->L[0].get(), {0, lw.first, 0}, lw.second);
    d->R[nsites].reset(make_tensor(ctx, {edge_bond(wl, TNX_BD_IN, q), redirected(wr, TNX_BD_IN),
                                         edge_bond(wl, TNX_BD_OUT, q)}));
    const auto rw = locate(wr, right_w);
    set_one(d->R[nsites].get(), {0, rw.first, 0}, rw.second);
    tnx_network* n = nullptr;
    chk(ctx, tnx_network_create(ctx, TWO_SITE, &n));
    d->two.reset(n);
    chk(ctx, tnx_network_create(ctx, HEFF, &n));
    d->heff.reset(n);
    chk(ctx, tnx_network_create(ctx, ENV_L, &n));
    d->envl.reset(n);
    chk(ctx, tnx_network_create(ctx, ENV_R, &n));
    d->envr.reset(n);
    for (tnx_network* x : {d->two.get(), d->envl.get(), d->envr.get()}) chk(ctx, tnx_network_set_order(x, 1, nullptr));
    chk(ctx, tnx_network_set_order(d->heff.get(), 2, nullptr));
    for (int i = nsites - 1; i >= 2; --i) env_right(d.get(), i);
    *out = d.release();
  });
}

extern "C" tnx_status tnx_dmrg_destroy(tnx_dmrg* d) {
  if (!d) return TNX_ERR_ARG;
  cudaStreamSynchronize(d->ctx->stream);
  delete d;
  return TNX_OK;
}

extern "C" tnx_status tnx_dmrg_sweep(tnx_dmrg* d, int64_t maxdim, double cutoff, int lanczos_steps, int prec,
                                     double* energy, double* max_trunc_err, int64_t* max_bond, double* phase_ms) {
  if (!d) return TNX_ERR_ARG;
  return tnx_guard(d->ctx, [&] {
    if (maxdim < 1 || lanczos_steps < 1) fail(TNX_ERR_ARG, "bad sweep arguments");
    tnx_ctx* c = d->ctx;
    chk(c, tnx_network_set_precision(d->heff.get(), prec));
    double ph[4] = {0, 0, 0, 0};   // two-site + Lanczos, SVD, environments, total
    const auto t_all = std::chrono::steady_clock::now();
    double lam = 0.0, terr_max = 0.0;
    int64_t bmax = 0;
    auto update = [&](int i, bool ltr) {
      auto t0 = std::chrono::steady_clock::now();
      TPtr psi(launch(d->two.get(), {{"A1", d->A[i].get()}, {"A2", d->A[i + 1].get()}}));
      TPtr evec(make_tensor(c, psi->bonds));
      for (auto& kv : std::vector<std::pair<const char*, tnx_tensor*>>{
               {"L", d->L[i].get()}, {"psi", psi.get()}, {"W1", d->W.get()}, {"W2", d->W.get()},
               {"R", d->R[i + 2].get()}})
        chk(c, tnx_network_put(d->heff.get(), kv.first, kv.second, 0, nullptr));
      int nmv = 0;
      chk(c, tnx_lanczos(d->heff.get(), "psi", psi.get(), lanczos_steps, &lam, evec.get(), &nmv));
      ph[0] += ms_since(t0);
      t0 = std::chrono::steady_clock::now();
      tnx_tensor *U = nullptr, *V = nullptr;
      double terr = 0.0, dw = 0.0;
      tnx_svd_run(evec.get(), 2, maxdim, cutoff, nullptr, 0, ltr ? 1 : 2, &U, nullptr, &V, &terr, &dw, nullptr);
      d->A[i].reset(U);
      d->A[i + 1].reset(V);
      terr_max = std::max(terr_max, terr);
      bmax = std::max(bmax, U->bonds.back().dim);
      ph[1] += ms_since(t0);
      t0 = std::chrono::steady_clock::now();
      if (ltr) env_left(d, i);
      else env_right(d, i + 1);
      ph[2] += ms_since(t0);
    };
    for (int i = 0; i + 1 < d->N; ++i) update(i, true);
    for (int i = d->N - 2; i >= 0; --i) update(i, false);
    ph[3] = ms_since(t_all);
    if (energy) *energy = lam;
    if (max_trunc_err) *max_trunc_err = terr_max;
    if (max_bond) *max_bond = bmax;
    if (phase_ms)
      for (int k = 0; k < 4; ++k) phase_ms[k] = ph[k];
  });
}

extern "C" tnx_status tnx_dmrg_tensor(const tnx_dmrg* d, int site, tnx_tensor** out) {
  if (!d) return TNX_ERR_ARG;
  return tnx_guard(d->ctx, [&] {
    if (!out || site < 0 || site >= d->N) fail(TNX_ERR_ARG, "bad site");
    tnx_tensor *a = nullptr, *b = nullptr;
    chk(d->ctx, tnx_tensor_dagger(d->A[site].get(), &a));
    TPtr tmp(a);
    chk(d->ctx, tnx_tensor_dagger(a, &b));
    *out = b;
  });
}
