// Dagger (Sec. 6.4) and the SVD of a block-sparse tensor with truncation
// (Sec. 9.1 / 9.2 of arXiv 2401.01921), on the device.
//
// The SVD maps the tensor to one dense matrix per total charge g of its row
// legs (the first `rowrank` legs): rows are the row-leg sector tuples of flux
// g in lexicographic order, each spanning the product of its degeneracies,
// columns likewise for the column legs.  The blocks are gathered into the
// Jacobi working layout (k_svd.cu), decomposed, and the singular values come
// back to the host, which applies the truncation rules of Svd_truncate: all
// values sorted together, the largest keepdim kept, values below err dropped,
// min_blockdim values per block of S kept regardless (they count towards
// keepdim; ties are ranked by block, then position).  The kept triplets are
// written into new block-sparse tensors U (row legs + a new OUT leg whose
// sectors are the kept charges, ascending), S (diagonal) and V^dagger (the new
// IN leg + the column legs).
#include <algorithm>
#include <numeric>

#include "tnx_plan.h"

namespace {

std::vector<int32_t> legs_flux(const std::vector<BondD>& bonds, const int32_t* q, int l0, int l1) {
  const int nsym = bonds.empty() ? 0 : bonds[0].nsym;
  std::vector<int32_t> f(nsym, 0);
  for (int l = l0; l < l1; ++l)
    for (int c = 0; c < nsym; ++c) f[c] += bonds[l].signed_q(q[l], c);
  for (int c = 0; c < nsym; ++c) {
    const int n = bonds[0].kinds[c] == TNX_ZN ? bonds[0].zn[c] : 0;
    if (n > 0) f[c] = ((f[c] % n) + n) % n;
  }
  return f;
}

int64_t tuple_dim(const std::vector<BondD>& bonds, const std::vector<int32_t>& t, int l0) {
  int64_t d = 1;
  for (size_t i = 0; i < t.size(); ++i) d *= bonds[l0 + i].deg[t[i]];
  return d;
}

struct Group {
  std::vector<int32_t> charge;
  std::map<std::vector<int32_t>, int64_t> rows, cols;   // tuple -> offset (filled in order)
  int64_t m = 0, n = 0;
  bool cols_are_vectors = true;
  int c = 0, r = 0;
  int64_t offX = 0, offJ = 0, offS = 0;
  std::vector<int> order;    // vector indices by descending sigma
  int kept = 0, forced = 0;
};

}  // namespace

extern "C" tnx_status tnx_tensor_dagger(const tnx_tensor* t, tnx_tensor** out) {
  if (!t) return TNX_ERR_ARG;
  return tnx_guard(t->ctx, [&] {
    if (!out) fail(TNX_ERR_ARG, "null output");
    std::vector<BondD> bs = t->bonds;
    for (auto& b : bs) b.dir = -b.dir;
    std::unique_ptr<tnx_tensor> r(make_tensor(t->ctx, bs));
    // reversing every leg negates the flux of every block: the stored blocks
    // and their order are the same
    if (r->nelem != t->nelem || r->nblk != t->nblk) fail(TNX_ERR_ARG, "internal: dagger changed the blocks");
    if (t->nelem > 0)
      CUDA_CHECK(cudaMemcpyAsync(r->data, t->data, (size_t)t->nelem * sizeof(double), cudaMemcpyDeviceToDevice,
                                 t->ctx->stream));
    else if (t->rank == 0)
      CUDA_CHECK(cudaMemcpyAsync(r->data, t->data, sizeof(double), cudaMemcpyDeviceToDevice, t->ctx->stream));
    *out = r.release();
  });
}

// Shared by the C-ABI call and the DMRG sweep.  Returns the new tensors; any
// of S_out may be null when not wanted (absorb != 0).
void tnx_svd_run(tnx_tensor* t, int rowrank, int64_t keepdim, double err, const int64_t* min_blockdim, int nmin,
                 int absorb, tnx_tensor** U_out, tnx_tensor** S_out, tnx_tensor** V_out, double* trunc_err,
                 double* discarded, int* sweeps_out) {
  tnx_ctx* ctx = t->ctx;
  cudaStream_t st = ctx->stream;
  const int R = t->rank;
  if (rowrank < 1 || rowrank >= R) fail(TNX_ERR_ARG, "rowrank must leave at least one row and one column leg");
  if (absorb < 0 || absorb > 2) fail(TNX_ERR_ARG, "absorb must be 0, 1 or 2");
  if (!U_out || !V_out || (absorb == 0 && !S_out)) fail(TNX_ERR_ARG, "null output");
  if (t->nblk == 0) fail(TNX_ERR_ARG, "the tensor stores no block");
  // ---- charge groups of the matrix form
  std::map<std::vector<int32_t>, Group> gm;
  for (int64_t b = 0; b < t->nblk; ++b) {
    const int32_t* q = t->qn.data() + (size_t)b * R;
    std::vector<int32_t> g = legs_flux(t->bonds, q, 0, rowrank);
    Group& G = gm[g];
    G.charge = g;
    G.rows[std::vector<int32_t>(q, q + rowrank)] = 0;
    G.cols[std::vector<int32_t>(q + rowrank, q + R)] = 0;
  }
  std::vector<Group*> groups;
  for (auto& kv : gm) groups.push_back(&kv.second);
  const int ngr = (int)groups.size();
  if (min_blockdim && nmin != ngr)
    fail(TNX_ERR_ARG, "min_blockdim needs one entry per block of S (" + std::to_string(ngr) + ")");
  int64_t nX = 0, nJ = 0, nS = 0;
  for (Group* G : groups) {
    for (auto& kv : G->rows) { kv.second = G->m; G->m += tuple_dim(t->bonds, kv.first, 0); }
    for (auto& kv : G->cols) { kv.second = G->n; G->n += tuple_dim(t->bonds, kv.first, rowrank); }
    G->cols_are_vectors = G->n <= G->m;
    const int64_t c = std::min(G->m, G->n), r = std::max(G->m, G->n);
    if (r > INT32_MAX / 2 || c > 65536) fail(TNX_ERR_UNSUPPORTED, "SVD block above 65536 x 2^30");
    G->c = (int)c;
    G->r = (int)r;
    G->offX = nX;
    G->offJ = nJ;
    G->offS = nS;
    nX += (c * r + 31) / 32 * 32;
    nJ += (c * c + 31) / 32 * 32;
    nS += (c + 31) / 32 * 32;
  }
  DevBuf X(ctx, (size_t)std::max<int64_t>(nX, 1) * 8), J(ctx, (size_t)std::max<int64_t>(nJ, 1) * 8),
      SG(ctx, (size_t)std::max<int64_t>(nS, 1) * 8), MO(ctx, 256);
  double* dX = (double*)X.p;
  double* dJ = (double*)J.p;
  double* dS = (double*)SG.p;
  std::vector<SvdGroup> hg(ngr);
  std::vector<int2> slots, vecs;
  int maxcp = 0, maxr = 0;
  for (int i = 0; i < ngr; ++i) {
    Group* G = groups[i];
    hg[i] = SvdGroup{dX + G->offX, dJ + G->offJ, dS + G->offS, G->c, G->r};
    const int cp = G->c + (G->c & 1);
    maxcp = std::max(maxcp, cp);
    maxr = std::max(maxr, G->r);   // r >= c
    for (int s = 0; s < cp / 2; ++s) slots.push_back(make_int2(i, s));
    for (int p = 0; p < G->c; ++p) vecs.push_back(make_int2(i, p));
  }
  // ---- gather the blocks into the working vectors
  std::vector<Copy2D> gather;
  for (int64_t b = 0; b < t->nblk; ++b) {
    const int32_t* q = t->qn.data() + (size_t)b * R;
    Group& G = gm[legs_flux(t->bonds, q, 0, rowrank)];
    const std::vector<int32_t> rt(q, q + rowrank), ct(q + rowrank, q + R);
    const int64_t r0 = G.rows[rt], c0 = G.cols[ct];
    const int64_t mt = tuple_dim(t->bonds, rt, 0), nt = tuple_dim(t->bonds, ct, rowrank);
    if (mt == 0 || nt == 0) continue;
    if (mt > INT32_MAX || nt > INT32_MAX) fail(TNX_ERR_UNSUPPORTED, "block above 2^31 rows or columns");
    Copy2D c;
    memset(&c, 0, sizeof(c));
    c.src = t->data + t->off[b];
    c.sld = nt;
    c.rows = (int32_t)mt;
    c.cols = (int32_t)nt;
    double* Xg = dX + G.offX;
    if (G.cols_are_vectors) {   // X = M^T: X[c0 + j][r0 + i]
      c.dst = Xg + c0 * G.r + r0;
      c.dld = G.r;
      c.trans = 1;
    } else {                    // X = M: X[r0 + i][c0 + j]
      c.dst = Xg + r0 * G.r + c0;
      c.dld = G.r;
      c.trans = 0;
    }
    gather.push_back(c);
  }
  std::vector<std::unique_ptr<DevBuf>> tmp;
  auto up = [&](const void* src, size_t bytes) {
    tmp.emplace_back(new DevBuf(ctx, std::max<size_t>(bytes, 256)));
    if (bytes) CUDA_CHECK(cudaMemcpyAsync(tmp.back()->p, src, bytes, cudaMemcpyHostToDevice, st));
    return tmp.back()->p;
  };
  const SvdGroup* dg = (const SvdGroup*)up(hg.data(), hg.size() * sizeof(SvdGroup));
  const int2* dslots = (const int2*)up(slots.data(), slots.size() * sizeof(int2));
  const int2* dvecs = (const int2*)up(vecs.data(), vecs.size() * sizeof(int2));
  const Copy2D* dgather = (const Copy2D*)up(gather.data(), gather.size() * sizeof(Copy2D));
  CUDA_CHECK(cudaMemsetAsync(dX, 0, (size_t)std::max<int64_t>(nX, 1) * 8, st));
  CUDA_CHECK(tnx_launch_copy2d(dgather, (int)gather.size(), st));
  constexpr int MAX_SWEEPS = 60;
  const int rounds = maxcp - 1;
  int sweeps = 0;
  bool done = rounds <= 0, via_qr = false;
  // ---- blocks of 16 or more vectors: QR-preconditioned Jacobi (k_svd.cu), the
  // pivoted QR and the sweeps on R each in one cooperative launch
  int maxc = 0;
  int64_t nC = 0, nC2 = 0, nCR = 0;
  for (Group* G : groups) {
    maxc = std::max(maxc, G->c);
    nC += (G->c + 31) / 32 * 32;
    nC2 += ((int64_t)G->c * G->c + 31) / 32 * 32;
    nCR += ((int64_t)G->c * G->r + 31) / 32 * 32;
  }
  std::unique_ptr<DevBuf> QD, QI, QXf;
  if (!done && maxc >= 16) {
    QD.reset(new DevBuf(ctx, (size_t)(3 * nC + 2 * nC2) * 8));   // tau, nrm[2], Xr, Jr
    QI.reset(new DevBuf(ctx, (size_t)(3 * nC) * 4));             // perm, pos[2]
    QXf.reset(new DevBuf(ctx, (size_t)std::max<int64_t>(nCR, 1) * 8));
    std::vector<SvdQr> hq(ngr);
    std::vector<SvdGroup> hr(ngr);
    std::vector<int2> qslots;
    int64_t oc = 0, oc2 = 0, ocr = 0;
    for (int i = 0; i < ngr; ++i) {
      Group* G = groups[i];
      SvdQr& q = hq[i];
      q.X = dX + G->offX;
      q.tau = (double*)QD->p + oc;
      q.nrm = (double*)QD->p + nC + 2 * oc;
      q.Xr = (double*)QD->p + 3 * nC + oc2;
      q.Jr = (double*)QD->p + 3 * nC + nC2 + oc2;
      q.perm = (int32_t*)QI->p + oc;
      q.pos = (int32_t*)QI->p + nC + 2 * oc;
      q.Xf = (double*)QXf->p + ocr;
      q.J = dJ + G->offJ;
      q.sigma = dS + G->offS;
      q.c = G->c;
      q.r = G->r;
      hr[i] = SvdGroup{q.Xr, q.Jr, q.sigma, G->c, G->c};
      for (int j = 0; j < G->c; ++j) qslots.push_back(make_int2(i, j));
      oc += (G->c + 31) / 32 * 32;
      oc2 += ((int64_t)G->c * G->c + 31) / 32 * 32;
      ocr += ((int64_t)G->c * G->r + 31) / 32 * 32;
    }
    const SvdQr* dq = (const SvdQr*)up(hq.data(), hq.size() * sizeof(SvdQr));
    const SvdGroup* dr = (const SvdGroup*)up(hr.data(), hr.size() * sizeof(SvdGroup));
    const int2* dqs = (const int2*)up(qslots.data(), qslots.size() * sizeof(int2));
    // [QR barrier count | QR status, pad | offmax per sweep | Jacobi barrier count | Jacobi status, sweeps]
    std::vector<uint64_t> zero(MAX_SWEEPS + 4, 0);
    unsigned long long* w = (unsigned long long*)up(zero.data(), zero.size() * 8);
    int* qstat = (int*)(w + 1);
    int* jstat = (int*)(w + MAX_SWEEPS + 3);
    const cudaError_t ce = tnx_launch_qr_coop(dq, dqs, (int)qslots.size(), maxc, w, qstat, st);
    if (ce == cudaSuccess) {
      CUDA_CHECK(tnx_launch_qr_gather_r(dq, ngr, maxc, st));
      // the sweeps run on R: vectors of c entries
      CUDA_CHECK(tnx_launch_jacobi_coop(dr, dslots, (int)slots.size(), maxcp, maxc, MAX_SWEEPS, 1e-13, w + 2,
                                        w + MAX_SWEEPS + 2, jstat, jstat + 1, st));
      CUDA_CHECK(tnx_launch_qr_apply(dq, dvecs, (int)vecs.size(), maxr, st));
      int hs[4] = {0, 0, 0, 0};
      CUDA_CHECK(cudaMemcpyAsync(hs, qstat, 4, cudaMemcpyDeviceToHost, st));
      CUDA_CHECK(cudaMemcpyAsync(hs + 2, jstat, 8, cudaMemcpyDeviceToHost, st));
      CUDA_CHECK(cudaStreamSynchronize(st));
      if (hs[0] != 0 || hs[2] != 0) fail(TNX_ERR_TIMEOUT, "SVD: a grid barrier of the QR or the Jacobi sweeps timed out");
      sweeps = hs[3];
      for (int i = 0; i < ngr; ++i) hg[i].X = hq[i].Xf;   // the extraction reads sigma_p u_p from Xf
      done = via_qr = true;
    } else if (ce == cudaErrorNotSupported || ce == cudaErrorCooperativeLaunchTooLarge) {
      (void)cudaGetLastError();   // the plain path below
    } else {
      CUDA_CHECK(ce);
    }
  }
  if (!via_qr) CUDA_CHECK(tnx_launch_jacobi_init(dg, ngr, st));
  // ---- plain path: sweeps until the largest relative off-diagonal met in a
  // sweep is small: one cooperative launch for everything; without it, one
  // launch per round
  if (!done) {
    // [offmax per sweep (8 B each) | barrier arrival count (8 B) | status | sweeps]
    std::vector<uint64_t> zero(MAX_SWEEPS + 2, 0);
    unsigned long long* w = (unsigned long long*)up(zero.data(), zero.size() * 8);
    unsigned long long* bar = w + MAX_SWEEPS;
    int* cstat = (int*)(w + MAX_SWEEPS + 1);
    const cudaError_t ce = tnx_launch_jacobi_coop(dg, dslots, (int)slots.size(), maxcp, maxr, MAX_SWEEPS, 1e-13, w,
                                                  bar, cstat, cstat + 1, st);
    if (ce == cudaSuccess) {
      int hs[2] = {0, 0};
      CUDA_CHECK(cudaMemcpyAsync(hs, cstat, sizeof(hs), cudaMemcpyDeviceToHost, st));
      CUDA_CHECK(cudaStreamSynchronize(st));
      if (hs[0] != 0) fail(TNX_ERR_TIMEOUT, "SVD: a grid barrier of the Jacobi sweeps timed out");
      sweeps = hs[1];
      done = true;
    } else if (ce == cudaErrorNotSupported || ce == cudaErrorCooperativeLaunchTooLarge) {
      (void)cudaGetLastError();   // the per-round path below
    } else {
      CUDA_CHECK(ce);
    }
  }
  unsigned long long* dmax = (unsigned long long*)MO.p;
  unsigned long long* hmax = (unsigned long long*)ctx->pinned;
  for (; !done && sweeps < MAX_SWEEPS; ++sweeps) {
    CUDA_CHECK(cudaMemsetAsync(dmax, 0, 8, st));
    for (int k = 0; k < rounds; ++k)
      CUDA_CHECK(tnx_launch_jacobi_round(dg, dslots, (int)slots.size(), k, dmax, st));
    CUDA_CHECK(cudaMemcpyAsync(hmax, dmax, 8, cudaMemcpyDeviceToHost, st));
    CUDA_CHECK(cudaStreamSynchronize(st));
    double off;
    memcpy(&off, hmax, 8);
    if (off <= 1e-13) {
      ++sweeps;
      break;
    }
  }
  if (sweeps_out) *sweeps_out = sweeps;
  if (!via_qr) CUDA_CHECK(tnx_launch_vector_norms(dg, dvecs, (int)vecs.size(), st));
  std::vector<double> sig((size_t)std::max<int64_t>(nS, 1));
  CUDA_CHECK(cudaMemcpyAsync(sig.data(), dS, (size_t)std::max<int64_t>(nS, 1) * 8, cudaMemcpyDeviceToHost, st));
  CUDA_CHECK(cudaStreamSynchronize(st));
  // ---- truncation (Svd_truncate rules)
  struct Cand {
    double s;
    int g, pos;
  };
  std::vector<Cand> rest;
  for (int i = 0; i < ngr; ++i) {
    Group* G = groups[i];
    const double* s = sig.data() + G->offS;
    G->order.resize(G->c);
    std::iota(G->order.begin(), G->order.end(), 0);
    std::stable_sort(G->order.begin(), G->order.end(), [&](int a, int b) { return s[a] > s[b]; });
    G->forced = min_blockdim ? (int)std::min<int64_t>(std::max<int64_t>(min_blockdim[i], 0), G->c) : 0;
    G->kept = G->forced;
    for (int k = G->forced; k < G->c; ++k) rest.push_back(Cand{s[G->order[k]], i, k});
  }
  std::stable_sort(rest.begin(), rest.end(), [](const Cand& a, const Cand& b) {
    if (a.s != b.s) return a.s > b.s;
    if (a.g != b.g) return a.g < b.g;
    return a.pos < b.pos;
  });
  int64_t forced_total = 0;
  for (Group* G : groups) forced_total += G->forced;
  const int64_t budget = keepdim > 0 ? std::max<int64_t>(keepdim - forced_total, 0) : INT64_MAX;
  int64_t taken = 0;
  size_t stop = rest.size();
  for (size_t x = 0; x < rest.size(); ++x) {
    if (rest[x].s < err || taken >= budget) {
      stop = x;
      break;
    }
    groups[rest[x].g]->kept++;
    ++taken;
  }
  double terr = 0.0, wsum = 0.0;
  for (size_t x = stop; x < rest.size(); ++x) {
    terr = std::max(terr, rest[x].s);
    wsum += rest[x].s * rest[x].s;
  }
  if (trunc_err) *trunc_err = terr;
  if (discarded) *discarded = wsum;
  // ---- the new bond and the output tensors
  const BondD& b0 = t->bonds[0];
  BondD cb;
  cb.nsym = b0.nsym;
  cb.kinds = b0.kinds;
  cb.zn = b0.zn;
  std::vector<int> newsec(ngr, -1);
  for (int i = 0; i < ngr; ++i) {
    Group* G = groups[i];
    if (G->kept == 0) continue;
    newsec[i] = cb.nsec++;
    cb.qn.insert(cb.qn.end(), G->charge.begin(), G->charge.end());
    cb.deg.push_back(G->kept);
  }
  if (cb.nsec == 0) fail(TNX_ERR_ARG, "the truncation keeps no singular value");
  if (b0.nsym == 0 && cb.nsec != 1) fail(TNX_ERR_ARG, "internal: a plain tensor gave several SVD blocks");
  BondD c_out = cb, c_in = cb;
  c_out.dir = b0.nsym ? TNX_BD_OUT : TNX_BD_REG;
  c_in.dir = b0.nsym ? TNX_BD_IN : TNX_BD_REG;
  c_out.finish();
  c_in.finish();
  std::vector<BondD> ub(t->bonds.begin(), t->bonds.begin() + rowrank), vb{c_in};
  ub.push_back(c_out);
  vb.insert(vb.end(), t->bonds.begin() + rowrank, t->bonds.end());
  std::unique_ptr<tnx_tensor> U(make_tensor(ctx, ub)), V(make_tensor(ctx, vb)), S;
  if (S_out) S.reset(make_tensor(ctx, {c_in, c_out}));
  // staging: U_g (m x kept) and V^T_g (kept x n) per kept group
  int64_t nU = 0, nV = 0;
  std::vector<int64_t> offU(ngr, 0), offV(ngr, 0);
  for (int i = 0; i < ngr; ++i) {
    offU[i] = nU;
    offV[i] = nV;
    nU += (groups[i]->m * groups[i]->kept + 31) / 32 * 32;
    nV += (groups[i]->n * groups[i]->kept + 31) / 32 * 32;
  }
  DevBuf UG(ctx, (size_t)std::max<int64_t>(nU, 1) * 8), VG(ctx, (size_t)std::max<int64_t>(nV, 1) * 8);
  std::vector<SvdOut> outs;
  for (int i = 0; i < ngr; ++i) {
    Group* G = groups[i];
    if (!G->kept) continue;
    double* Sblk = nullptr;
    if (S) {
      const std::vector<int32_t> key{newsec[i], newsec[i]};
      Sblk = S->data + S->off[S->index.at(key)];
    }
    for (int k = 0; k < G->kept; ++k) {
      SvdOut o;
      memset(&o, 0, sizeof(o));
      o.g = hg[i];
      o.p = G->order[k];
      o.k = k;
      o.absorb = absorb;
      o.cols_are_vectors = G->cols_are_vectors ? 1 : 0;
      o.U = (double*)UG.p + offU[i];
      o.ldu = G->kept;
      o.Vt = (double*)VG.p + offV[i];
      o.ldv = G->n;
      o.S = Sblk;
      o.lds = G->kept;
      outs.push_back(o);
    }
  }
  std::vector<Copy2D> scatter;
  for (int64_t b = 0; b < U->nblk; ++b) {
    const int32_t* q = U->qn.data() + (size_t)b * (rowrank + 1);
    const int gi = (int)std::distance(gm.begin(), gm.find(legs_flux(t->bonds, q, 0, rowrank)));
    Group* G = groups[gi];
    const std::vector<int32_t> rt(q, q + rowrank);
    const int64_t r0 = G->rows.at(rt), mt = tuple_dim(t->bonds, rt, 0);
    if (!mt) continue;
    Copy2D c;
    memset(&c, 0, sizeof(c));
    c.src = (double*)UG.p + offU[gi] + r0 * G->kept;
    c.dst = U->data + U->off[b];
    c.sld = c.dld = G->kept;
    c.rows = (int32_t)mt;
    c.cols = G->kept;
    scatter.push_back(c);
  }
  for (int64_t b = 0; b < V->nblk; ++b) {
    const int32_t* q = V->qn.data() + (size_t)b * (R - rowrank + 1);
    int gi = -1;
    for (int i = 0; i < ngr; ++i)
      if (newsec[i] == q[0]) gi = i;
    Group* G = groups[gi];
    const std::vector<int32_t> ct(q + 1, q + 1 + (R - rowrank));
    const int64_t c0 = G->cols.at(ct), nt = tuple_dim(t->bonds, ct, rowrank);
    if (!nt) continue;
    Copy2D c;
    memset(&c, 0, sizeof(c));
    c.src = (double*)VG.p + offV[gi] + c0;
    c.dst = V->data + V->off[b];
    c.sld = G->n;
    c.dld = nt;
    c.rows = G->kept;
    c.cols = (int32_t)nt;
    scatter.push_back(c);
  }
  const SvdOut* douts = (const SvdOut*)up(outs.data(), outs.size() * sizeof(SvdOut));
  const Copy2D* dsc = (const Copy2D*)up(scatter.data(), scatter.size() * sizeof(Copy2D));
  CUDA_CHECK(tnx_launch_svd_extract(douts, (int)outs.size(), st));
  CUDA_CHECK(tnx_launch_copy2d(dsc, (int)scatter.size(), st));
  CUDA_CHECK(cudaStreamSynchronize(st));   // the staging buffers are released on return
  *U_out = U.release();
  *V_out = V.release();
  if (S_out) *S_out = S.release();
}

extern "C" tnx_status tnx_svd_truncate(tnx_tensor* t, int rowrank, int64_t keepdim, double err,
                                       const int64_t* min_blockdim, int nmin, int absorb, tnx_tensor** U,
                                       tnx_tensor** S, tnx_tensor** Vdag, double* trunc_err, double* discarded) {
  if (!t) return TNX_ERR_ARG;
  return tnx_guard(t->ctx, [&] {
    tnx_svd_run(t, rowrank, keepdim, err, min_blockdim, nmin, absorb, U, S, Vdag, trunc_err, discarded, nullptr);
  });
}
