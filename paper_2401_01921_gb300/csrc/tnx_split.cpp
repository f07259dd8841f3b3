// Split-precision planning: per pairwise step, the row-exponent and slicing
// jobs that turn the packed FP64 operands into tiles of integer-valued 16-bit
// slices, and the tile list of the tcgen05 split GEMM (k_split.cu).  The
// one-pass TF32 variant uses the same plan with one slice of FP32 words per
// operand (16 K values, 64 bytes, per tile row: the same bytes per tile).
#include <algorithm>
#include <queue>

#include "tnx_plan.h"


namespace {
constexpr int TM = 128, TK = 32;
constexpr int64_t KMAX = 8192;   // the 64-bit fixed-point accumulator is exact up to this K
}

// Work items of one slicing launch (k_split.cu), one CTA (8 warps) each: a
// job gives each 8-row group 1, 2, 4 or 8 warps by the number of its 32-wide
// K tiles (a warp then takes about two of them, at most every eighth), and an
// item holds 8 / wpg consecutive groups of one job.
std::vector<int2> tnx_slice_schedule(std::vector<SliceJob>& jobs) {
  std::vector<int2> items;
  for (size_t q = 0; q < jobs.size(); ++q) {
    SliceJob& j = jobs[q];
    const int KT = (j.K + TK - 1) / TK;
    j.wpg = KT >= 16 ? 8 : KT >= 8 ? 4 : KT >= 3 ? 2 : 1;
    const int64_t g = ((int64_t)j.rows + j.tile_rows - 1) / j.tile_rows * (j.tile_rows / 8);
    if (g > INT32_MAX) fail(TNX_ERR_UNSUPPORTED, "slicing job above 2^31 row groups");
    for (int64_t r = 0; r < g; r += 8 / j.wpg) items.push_back(make_int2((int)q, (int)r));
  }
  return items;
}

// TF32 rows: every job one warp per 8-row group, eight groups per CTA item.
std::vector<int2> tnx_tf32_schedule(std::vector<SliceJob>& jobs) {
  std::vector<int2> items;
  for (size_t q = 0; q < jobs.size(); ++q) {
    SliceJob& j = jobs[q];
    j.wpg = 1;
    const int64_t g = ((int64_t)j.rows + j.tile_rows - 1) / j.tile_rows * (j.tile_rows / 8);
    if (g > INT32_MAX) fail(TNX_ERR_UNSUPPORTED, "TF32 operand above 2^31 row groups");
    for (int64_t r = 0; r < g; r += 8) items.push_back(make_int2((int)q, (int)r));
  }
  return items;
}

void tnx_build_split_parts(Plan& p, StepPlan& s) {
  const bool tf32 = p.prec == TNX_PREC_TF32;
  const int G = s.G;
  const int n = tf32 ? 1 : p.nslice;
  const int TKE = tf32 ? 16 : TK;   // K values per 64-byte tile row
  std::vector<SliceJob> jobs[2];
  int64_t elems[2] = {0, 0};
  std::vector<int64_t> offSA(G), offSB(G), offEA(G), offEB(G), offKX(G, 0);
  int64_t sa = 0, sb = 0, ea = 0, eb = 0, kx = 0;
  // Tile width: 32 columns when the 32-wide tiles of the step fit in one wave
  // on the 152 SMs (the CTAs then take half the columns each, which halves
  // their drain and conversion), else 64.
  int64_t tiles32 = 0;
  for (int g = 0; g < G; ++g)
    if (!s.skinny[g]) tiles32 += (s.mkn[3 * g] + TM - 1) / TM * ((s.mkn[3 * g + 2] + 31) / 32);
  const int TN = (p.narrow_tiles && tiles32 <= 152) ? 32 : 64;
  s.split_tn = TN;
  for (int g = 0; g < G; ++g) {
    const int64_t M = s.mkn[3 * g], K = s.mkn[3 * g + 1], N = s.mkn[3 * g + 2];
    if (s.skinny[g]) {
      offSA[g] = sa;
      offSB[g] = sb;
      offEA[g] = ea;
      offEB[g] = eb;
      continue;
    }
    if (K > KMAX) fail(TNX_ERR_UNSUPPORTED, "split precision supports K <= 8192 per charge sector");
    s.split_kmax = (int)std::max<int64_t>(s.split_kmax, K);
    const int64_t KT = (K + TKE - 1) / TKE, MT = (M + TM - 1) / TM, NT = (N + TN - 1) / TN;
    offSA[g] = sa;
    offSB[g] = sb;
    offEA[g] = ea;
    offEB[g] = eb;
    offKX[g] = kx;
    kx += KT * TKE;
    sa += MT * KT * n * (int64_t)(TM * TK * 2);
    sb += NT * KT * n * (int64_t)(TN * TK * 2);
    ea += M;
    eb += N;
  }
  s.slotSA = p.new_slot(p.alloc_zero((size_t)sa), sa / 8);
  s.slotSB = p.new_slot(p.alloc_zero((size_t)sb), sb / 8);
  s.slotEA = p.new_slot(p.alloc_zero((size_t)std::max<int64_t>(ea, 1) * 4), ea / 2);
  s.slotEB = p.new_slot(p.alloc_zero((size_t)std::max<int64_t>(eb, 1) * 4), eb / 2);
  if (!tf32) s.slotKX = p.new_slot(p.alloc_zero((size_t)std::max<int64_t>(kx, 1) * 4), kx / 2);
  for (int side = 0; side < 2; ++side) {
    for (int g = 0; g < G; ++g) {
      if (s.skinny[g]) continue;
      const int64_t M = s.mkn[3 * g], K = s.mkn[3 * g + 1], N = s.mkn[3 * g + 2];
      SliceJob j;
      memset(&j, 0, sizeof(j));
      const int64_t rows = side == 0 ? M : N;
      const int tr = side == 0 ? TM : TN;
      j.src_slot = side == 0 ? s.slotA : s.slotB;
      j.src_off = side == 0 ? s.offA[g] : s.offB[g];
      j.dst_slot = side == 0 ? s.slotSA : s.slotSB;
      j.dst_off_bytes = side == 0 ? offSA[g] : offSB[g];
      j.exp_slot = side == 0 ? s.slotEA : s.slotEB;
      j.exp_off = side == 0 ? offEA[g] : offEB[g];
      j.rows = (int32_t)rows;
      j.K = (int32_t)K;
      j.ld = (int32_t)s.ldK[g];
      j.tile_rows = tr;
      j.kx_slot = tf32 ? -1 : s.slotKX;
      j.kx_off = offKX[g];
      j.kx_sign = side == 0 ? -1 : 1;   // A's columns scaled down, B's rows up
      jobs[side].push_back(j);
      elems[side] += rows * K;
    }
  }
  auto make = [&](std::vector<SliceJob> js, int64_t el) {
    const std::vector<int2> items = tf32 ? tnx_tf32_schedule(js) : tnx_slice_schedule(js);
    StepPlan::Jobs J;
    J.n = (int)js.size();
    J.nitems = (int64_t)items.size();
    J.elems = el;
    J.d = p.upload(js);
    J.items = p.upload(items);
    J.h = js;
    return J;
  };
  if (!tf32) {
    std::vector<KexpJob> kj;
    for (int g = 0; g < G; ++g) {
      if (s.skinny[g]) continue;
      KexpJob k;
      memset(&k, 0, sizeof(k));
      k.src_slot = s.slotA;
      k.src_off = s.offA[g];
      k.kx_slot = s.slotKX;
      k.kx_off = offKX[g];
      k.rows = (int32_t)s.mkn[3 * g];
      k.K = (int32_t)s.mkn[3 * g + 1];
      k.ld = (int32_t)s.ldK[g];
      kj.push_back(k);
    }
    const std::vector<int4> ki = tnx_kexp_items(kj);
    s.dKJ = p.upload(kj);
    s.nkj = (int)kj.size();
    s.dKI = p.upload(ki);
    s.nki = (int64_t)ki.size();
    s.hKJ = kj;
  }
  std::vector<SliceJob> all = jobs[0];
  all.insert(all.end(), jobs[1].begin(), jobs[1].end());
  s.jobsA = make(jobs[0], elems[0]);
  s.jobsB = make(jobs[1], elems[1]);
  s.jobsAll = make(all, elems[0] + elems[1]);
  s.slice_elems = elems[0] + elems[1];
  std::vector<SplitGroup> sg(G);
  std::vector<GemmTile> tiles;
  for (int g = 0; g < G; ++g) {
    SplitGroup& x = sg[g];
    memset(&x, 0, sizeof(x));
    x.a_slot = s.slotSA;
    x.b_slot = s.slotSB;
    x.c_slot = s.slotC;
    x.ea_slot = s.slotEA;
    x.out_slot = -1;
    x.fc_slot = -1;
    x.eb_slot = s.slotEB;
    x.a_off_bytes = offSA[g];
    x.b_off_bytes = offSB[g];
    x.c_off = s.offC[g];
    x.ea_off = offEA[g];
    x.eb_off = offEB[g];
    x.M = (int32_t)s.mkn[3 * g];
    x.K = (int32_t)s.mkn[3 * g + 1];
    x.N = (int32_t)s.mkn[3 * g + 2];
    x.ldc = x.N;
    if (s.skinny[g]) continue;
    // Tiles that run at the same time should share the larger operand panel,
    // so that the smaller one is what gets re-read (from L2): column-major
    // order (tiles of one B column panel together) when A is the smaller.
    if (x.M < x.N) {
      for (int n0 = 0; n0 < x.N; n0 += TN)
        for (int m0 = 0; m0 < x.M; m0 += TM) tiles.push_back(GemmTile{g, m0, n0, 0});
    } else {
      for (int m0 = 0; m0 < x.M; m0 += TM)
        for (int n0 = 0; n0 < x.N; n0 += TN) tiles.push_back(GemmTile{g, m0, n0, 0});
    }
  }
  std::stable_sort(tiles.begin(), tiles.end(),
                   [&](const GemmTile& x, const GemmTile& y) { return sg[x.group].K > sg[y.group].K; });
  // More tiles than SMs (one CTA fits per SM): a persistent grid of 152 CTAs,
  // each streaming its next tile's operands while it drains the current one.
  // Tiles go to CTAs longest first, each to the least loaded CTA (work = K
  // tiles plus a fixed drain cost); CTA c takes positions c, c + NC, ... of the
  // device list, and holes (group -1) pad the shorter lists.
  const int NC = (int)std::min<size_t>(tiles.size(), 152);
  std::vector<GemmTile> sched = tiles;
  if (NC > 0 && (size_t)NC < tiles.size()) {
    std::vector<std::vector<int>> per(NC);
    typedef std::pair<int64_t, int> Load;   // (work, cta)
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int c = 0; c < NC; ++c) heap.push(Load(0, c));
    for (size_t t = 0; t < tiles.size(); ++t) {
      Load l = heap.top();
      heap.pop();
      per[l.second].push_back((int)t);
      l.first += (sg[tiles[t].group].K + TKE - 1) / TKE + 4;
      heap.push(l);
    }
    size_t depth = 0;
    for (auto& v : per) depth = std::max(depth, v.size());
    sched.assign((size_t)NC * depth, GemmTile{-1, 0, 0, 0});
    for (int c = 0; c < NC; ++c)
      for (size_t k = 0; k < per[c].size(); ++k) sched[c + k * NC] = tiles[per[c][k]];
  }
  s.dSG = p.upload(sg);
  s.dST = p.upload(sched);
  s.nstiles = (int)sched.size();
  s.split_grid = NC;
  s.hSG = sg;
  s.hST = tiles;
}

// Work items of the K-balancing pass: 32 K indices by 64 rows each.
std::vector<int4> tnx_kexp_items(const std::vector<KexpJob>& jobs) {
  std::vector<int4> items;
  for (size_t q = 0; q < jobs.size(); ++q)
    for (int k0 = 0; k0 < jobs[q].K; k0 += 32)
      for (int r0 = 0; r0 < jobs[q].rows; r0 += 64) items.push_back(make_int4((int)q, k0, r0, 0));
  return items;
}

// balance: slice with K balancing.  The exponents come from A, so they are
// recomputed whenever A is re-prepared; a B re-prepared alone reuses them.
void tnx_enqueue_split(Plan& p, StepPlan& s, cudaStream_t st, bool needA, bool needB, bool balance) {
  const int f16 = p.prec == TNX_PREC_SPLIT_F16 ? 1 : 0;
  const StepPlan::Jobs* J = (needA && needB) ? &s.jobsAll : needA ? &s.jobsA : needB ? &s.jobsB : nullptr;
  if (p.prec == TNX_PREC_TF32) {
    if (J && J->n) {
      ProfScope ps(p.ctx, st, TNX_KC_SLICE, (double)J->elems * (8.0 + 8.0 + 4.0));
      CUDA_CHECK(tnx_launch_tf32_rows(J->d, J->items, J->nitems, p.d_slots, st));
    }
    ProfScope ps(p.ctx, st, TNX_KC_GEMM, s.flops - s.flops_skinny);
    CUDA_CHECK(tnx_launch_gemm_tf32(s.dSG, s.dST, s.nstiles, p.d_slots, p.ctx->d_status, st, s.split_grid,
                                    s.split_tn, s.split_fold ? 1 : 0));
    return;
  }
  if (J && J->n) {
    ProfScope ps(p.ctx, st, TNX_KC_SLICE, (double)J->elems * (8.0 + 8.0 + 2.0 * p.nslice));
    if (balance && needA) CUDA_CHECK(tnx_launch_kexp(s.dKJ, s.nkj, s.dKI, s.nki, p.d_slots, st));
    CUDA_CHECK(tnx_launch_slices(J->d, J->items, J->nitems, p.nslice, p.beta, f16, p.d_slots, st, balance ? 1 : 0));
  }
  ProfScope ps(p.ctx, st, TNX_KC_GEMM, s.flops - s.flops_skinny);
  CUDA_CHECK(tnx_launch_gemm_split(s.dSG, s.dST, s.nstiles, p.nslice, p.beta, f16, p.d_slots, p.ctx->d_status, st,
                                   s.split_grid, s.split_tn, s.split_fold ? 1 : s.split_kmax <= 160 ? 2 : 0));
}
