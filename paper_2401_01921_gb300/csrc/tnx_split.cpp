// Split-precision planning: per pairwise step, the row-exponent and slicing
// jobs that turn the packed FP64 operands into tiles of integer-valued 16-bit
// slices, and the tile list of the tcgen05 split GEMM (k_split.cu).
#include "tnx_plan.h"

size_t tnx_split_smem_bytes(int nslice);

namespace {
constexpr int TM = 128, TN = 64, TK = 32;
constexpr int64_t KMAX = 8192;   // the 64-bit fixed-point accumulator is exact up to this K
}

void tnx_build_split_parts(Plan& p, StepPlan& s) {
  if (p.prec == TNX_PREC_TF32) fail(TNX_ERR_UNSUPPORTED, "TF32 products are not available in this build");
  const int G = s.G;
  const int n = p.nslice;
  std::vector<SliceJob> jobs;
  std::vector<int64_t> row_start(1, 0), warp_start(1, 0);
  std::vector<int64_t> offSA(G), offSB(G), offEA(G), offEB(G);
  int64_t sa = 0, sb = 0, ea = 0, eb = 0;
  for (int g = 0; g < G; ++g) {
    const int64_t M = s.mkn[3 * g], K = s.mkn[3 * g + 1], N = s.mkn[3 * g + 2];
    if (K > KMAX) fail(TNX_ERR_UNSUPPORTED, "split precision supports K <= 8192 per charge sector");
    const int64_t KT = (K + TK - 1) / TK, MT = (M + TM - 1) / TM, NT = (N + TN - 1) / TN;
    offSA[g] = sa;
    offSB[g] = sb;
    offEA[g] = ea;
    offEB[g] = eb;
    sa += MT * KT * n * (int64_t)(TM * TK * 2);
    sb += NT * KT * n * (int64_t)(TN * TK * 2);
    ea += M;
    eb += N;
  }
  s.slotSA = p.new_slot(p.alloc_zero((size_t)sa), sa / 8);
  s.slotSB = p.new_slot(p.alloc_zero((size_t)sb), sb / 8);
  s.slotEA = p.new_slot(p.alloc_zero((size_t)std::max<int64_t>(ea, 1) * 4), ea / 2);
  s.slotEB = p.new_slot(p.alloc_zero((size_t)std::max<int64_t>(eb, 1) * 4), eb / 2);
  for (int side = 0; side < 2; ++side) {
    for (int g = 0; g < G; ++g) {
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
      const int64_t KT = (K + TK - 1) / TK;
      const int64_t padded = (rows + tr - 1) / tr * tr;
      jobs.push_back(j);
      row_start.push_back(row_start.back() + rows);
      warp_start.push_back(warp_start.back() + padded / 8 * KT);
    }
  }
  s.njobs = (int)jobs.size();
  s.totRows = row_start.back();
  s.totTiles = warp_start.back();
  s.dJobs = p.upload(jobs);
  s.dRowStart = p.upload(row_start);
  s.dTileStart = p.upload(warp_start);
  std::vector<SplitGroup> sg(G);
  std::vector<GemmTile> tiles;
  for (int g = 0; g < G; ++g) {
    SplitGroup& x = sg[g];
    memset(&x, 0, sizeof(x));
    x.a_slot = s.slotSA;
    x.b_slot = s.slotSB;
    x.c_slot = s.slotC;
    x.ea_slot = s.slotEA;
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
    for (int m0 = 0; m0 < x.M; m0 += TM)
      for (int n0 = 0; n0 < x.N; n0 += TN) tiles.push_back(GemmTile{g, m0, n0, 0});
  }
  s.dSG = p.upload(sg);
  s.dST = p.upload(tiles);
  s.nstiles = (int)tiles.size();
}

void tnx_enqueue_split(Plan& p, StepPlan& s, cudaStream_t st) {
  const int f16 = p.prec == TNX_PREC_SPLIT_F16 ? 1 : 0;
  const double elems = (double)(s.copyA.total + s.copyB.total);
  {
    ProfScope ps(p.ctx, st, TNX_KC_SLICE, elems * (8.0 + 8.0 + 2.0 * p.nslice));
    CUDA_CHECK(tnx_launch_row_exponents(s.dJobs, s.dRowStart, s.njobs, s.totRows, p.d_slots, st));
    CUDA_CHECK(tnx_launch_slices(s.dJobs, s.dTileStart, s.njobs, s.totTiles, p.nslice, p.beta, f16, p.d_slots, st));
  }
  ProfScope ps(p.ctx, st, TNX_KC_GEMM, s.flops);
  CUDA_CHECK(tnx_launch_gemm_split(s.dSG, s.dST, s.nstiles, p.nslice, p.beta, f16, p.d_slots, p.ctx->d_status, st));
}
