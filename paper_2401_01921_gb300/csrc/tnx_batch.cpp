// Batched contraction: many networks with the same blueprint and contraction
// tree run as one sequence of launches (one relayout launch and one grouped
// GEMM launch per pairwise step for all instances together), captured in one
// CUDA graph.  The split GEMM's launch schedule (one CTA per tile, or a
// persistent grid of 1x / 2x / 3x the SM count over a longest-K-first tile
// list) is picked by timing each candidate on the batch itself.
//
// Each instance keeps its own plan (tables, packed operands, intermediates);
// the batch only merges the task tables, shifting every slot index by the
// instance's offset in the merged slot table.  Instances whose plan fuses an
// MPO step (gather, skinny product, scatter in one kernel) keep it: their
// fused tiles join one fused launch and the relayouts it does are left out of
// the merged relayouts; the other instances' products run as skinny tiles.
#include <algorithm>
#include <cstring>

#include "tnx_plan.h"

Plan* tnx_ensure_plan(tnx_network* net);
void tnx_bind_inputs(tnx_network* net, Plan& p);
void tnx_check_out_bonds(const Plan& p, const tnx_tensor* out);
void tnx_capture_graph(tnx_ctx* c, cudaStream_t st, GraphRec& g, const std::function<void()>& body);

struct BStep {
  TaskList A, B;
  GemmGroup* dG = nullptr;
  GemmTile *dT = nullptr, *dTs = nullptr;
  int nt = 0, nts = 0;
  StepPlan::Jobs jobs;
  KexpJob* dKJ = nullptr;       // K balancing of the split steps (every launch: all operands are new)
  int nkj = 0;
  int4* dKI = nullptr;
  int64_t nki = 0;
  SplitGroup* dSG = nullptr;
  GemmTile* dST = nullptr;
  int nst = 0;
  int kmax = 0;                 // largest K of the merged split groups
  double flops = 0, flops_skinny = 0;
  // the fused MPO steps of the instances that fuse this step: merged tiles and
  // column descriptors (the other instances run copies and skinny tiles)
  FusedTile* dFT = nullptr;
  FusedCol* dFC = nullptr;
  int nft = 0, fkp = 0, fnp = 0;
};

struct tnx_batch {
  tnx_ctx* ctx = nullptr;
  std::vector<tnx_network*> nets;
  std::vector<uint64_t> serials;
  std::vector<Plan*> plans;
  std::vector<int> base;      // slot offset per instance
  int prec = TNX_PREC_F64, nslice = 6, beta = 7;
  std::vector<std::unique_ptr<DevBuf>> bufs;
  std::vector<double*> h_slots;
  double** d_slots = nullptr;
  std::vector<BStep> steps;
  TaskList fin;
  int split_grid = 0;
  std::unique_ptr<GraphRec> graph;

  template <class T>
  T* upload(const std::vector<T>& v) {
    size_t n = std::max<size_t>(v.size(), 1) * sizeof(T);
    bufs.emplace_back(new DevBuf(ctx, n));
    if (!v.empty())
      CUDA_CHECK(cudaMemcpyAsync(bufs.back()->p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return (T*)bufs.back()->p;
  }
};

namespace {

int shift_slot(int s, int b) { return s < 0 ? s : s + b; }

// parts: (instance, its task list) for the instances whose relayout runs
TaskList merge_tasks(tnx_batch& B, const std::vector<std::pair<int, const TaskList*>>& parts) {
  std::vector<CopyTask> tasks;
  std::vector<int4> chunks;
  TaskList out;
  // bands, which only pay off inside a fused step, go back to plain tasks
  // (small tasks of many instances pack together)
  for (const auto& pr : parts) {
    for (CopyTask t : tnx_unband_tasks(pr.second->h)) {
      t.src_slot = shift_slot(t.src_slot, B.base[pr.first]);
      t.dst_slot = shift_slot(t.dst_slot, B.base[pr.first]);
      tasks.push_back(t);
    }
    out.total += pr.second->total;
  }
  tnx_make_copy_chunks(tasks, chunks);   // small tasks of different instances pack together
  out.n = (int)tasks.size();
  out.nchunks = (int)chunks.size();
  out.d = B.upload(tasks);
  out.chunks = B.upload(chunks);
  return out;
}

void enqueue_batch(tnx_batch& B, cudaStream_t st) {
  tnx_ctx* c = B.ctx;
  const int f16 = B.prec == TNX_PREC_SPLIT_F16 ? 1 : 0;
  for (auto& s : B.steps) {
    // the relayout lists leave out what fused steps do (their gathers, and the
    // operands their scatters write)
    if (s.A.n || s.B.n) {
      ProfScope ps(c, st, TNX_KC_RELAYOUT, 16.0 * (double)(s.A.total + s.B.total));
      if (s.A.n) CUDA_CHECK(tnx_launch_copy(s.A.d, s.A.chunks, s.A.nchunks, B.d_slots, st));
      if (s.B.n) CUDA_CHECK(tnx_launch_copy(s.B.d, s.B.chunks, s.B.nchunks, B.d_slots, st));
    }
    if (s.nft) {
      ProfScope ps(c, st, TNX_KC_SKINNY, s.flops_skinny);
      CUDA_CHECK(tnx_launch_fused_skinny(s.dG, s.dFT, s.nft, s.dFC, s.fkp, s.fnp, B.d_slots, st));
    }
    if (s.nts) {
      ProfScope ps(c, st, TNX_KC_SKINNY, s.flops_skinny);
      CUDA_CHECK(tnx_launch_gemm_skinny(s.dG, s.dTs, s.nts, B.d_slots, st));
    }
    if (B.prec == TNX_PREC_F64 || B.prec == TNX_PREC_F32) {
      ProfScope ps(c, st, TNX_KC_GEMM, s.flops - s.flops_skinny);
      if (B.prec == TNX_PREC_F64) CUDA_CHECK(tnx_launch_gemm_f64(s.dG, s.dT, s.nt, B.d_slots, st));
      else CUDA_CHECK(tnx_launch_gemm_f32(s.dG, s.dT, s.nt, B.d_slots, st));
    } else if (B.prec == TNX_PREC_TF32) {
      if (s.jobs.n) {
        ProfScope ps(c, st, TNX_KC_SLICE, (double)s.jobs.elems * 20.0);
        CUDA_CHECK(tnx_launch_tf32_rows(s.jobs.d, s.jobs.items, s.jobs.nitems, B.d_slots, st));
      }
      ProfScope ps(c, st, TNX_KC_GEMM, s.flops - s.flops_skinny);
      CUDA_CHECK(tnx_launch_gemm_tf32(s.dSG, s.dST, s.nst, B.d_slots, c->d_status, st, B.split_grid, 64));
    } else {
      if (s.jobs.n) {
        ProfScope ps(c, st, TNX_KC_SLICE, (double)s.jobs.elems * (16.0 + 2.0 * B.nslice));
        CUDA_CHECK(tnx_launch_kexp(s.dKJ, s.nkj, s.dKI, s.nki, B.d_slots, st));
        CUDA_CHECK(tnx_launch_slices(s.jobs.d, s.jobs.items, s.jobs.nitems, B.nslice, B.beta, f16, B.d_slots, st, 1));
      }
      ProfScope ps(c, st, TNX_KC_GEMM, s.flops - s.flops_skinny);
      CUDA_CHECK(tnx_launch_gemm_split(s.dSG, s.dST, s.nst, B.nslice, B.beta, f16, B.d_slots, c->d_status, st,
                                       B.split_grid, 64, s.kmax <= 160 ? 2 : 0));
    }
  }
  ProfScope ps(c, st, TNX_KC_FINAL, 16.0 * (double)B.fin.total);
  CUDA_CHECK(tnx_launch_copy(B.fin.d, B.fin.chunks, B.fin.nchunks, B.d_slots, st));
}

void check_fresh(const tnx_batch& B) {
  for (size_t i = 0; i < B.nets.size(); ++i)
    if (!B.nets[i]->plan || B.nets[i]->plan->serial != B.serials[i])
      fail(TNX_ERR_ARG, "a network of the batch was re-planned since the batch was created; create a new batch");
}

void bind(tnx_batch& B, tnx_tensor* const* outs) {
  for (size_t i = 0; i < B.nets.size(); ++i) {
    Plan& p = *B.plans[i];
    tnx_check_out_bonds(p, outs[i]);
    tnx_bind_inputs(B.nets[i], p);
    p.h_slots[p.out_slot] = outs[i]->data;
    for (size_t k = 0; k < p.h_slots.size(); ++k) B.h_slots[B.base[i] + k] = p.h_slots[k];
  }
  CUDA_CHECK(cudaMemcpyAsync(B.d_slots, B.h_slots.data(), B.h_slots.size() * sizeof(double*), cudaMemcpyHostToDevice,
                             B.ctx->stream));
}

}  // namespace

extern "C" tnx_status tnx_batch_create(tnx_ctx* ctx, int n, tnx_network* const* nets, tnx_batch** out) {
  return tnx_guard(ctx, [&] {
    if (!ctx || n < 1 || !nets || !out) fail(TNX_ERR_ARG, "bad batch arguments");
    std::unique_ptr<tnx_batch> B(new tnx_batch());
    B->ctx = ctx;
    int slots = 0;
    for (int i = 0; i < n; ++i) {
      if (!nets[i] || nets[i]->ctx != ctx) fail(TNX_ERR_ARG, "every network must belong to the context");
      for (int j = 0; j < i; ++j)
        if (nets[j] == nets[i]) fail(TNX_ERR_ARG, "a network appears twice in the batch");
      // one merged launch needs one tile width: networks in a batch keep 64-wide split tiles
      nets[i]->narrow_tiles = false;
      Plan* p = tnx_ensure_plan(nets[i]);
      if (i > 0 && (p->steps.size() != B->plans[0]->steps.size() || p->prec != B->prec))
        fail(TNX_ERR_ARG, "batched networks need the same number of contractions and the same precision");
      B->nets.push_back(nets[i]);
      B->plans.push_back(p);
      B->serials.push_back(p->serial);
      B->prec = p->prec;
      B->nslice = p->nslice;
      B->beta = p->beta;
      B->base.push_back(slots);
      slots += (int)p->h_slots.size();
    }
    B->h_slots.assign(slots, nullptr);
    B->bufs.emplace_back(new DevBuf(ctx, (size_t)slots * sizeof(double*)));
    B->d_slots = (double**)B->bufs.back()->p;
    const size_t nst = B->plans[0]->steps.size();
    B->steps.resize(nst);
    const bool split = B->prec == TNX_PREC_SPLIT_BF16 || B->prec == TNX_PREC_SPLIT_F16 || B->prec == TNX_PREC_TF32;
    for (size_t s = 0; s < nst; ++s) {
      BStep& bs = B->steps[s];
      // per instance: a fused step gathers its A itself, and a relayout that a
      // fused step's scatter writes is left out
      std::vector<std::pair<int, const TaskList*>> pa, pb;
      for (size_t i = 0; i < B->plans.size(); ++i) {
        const StepPlan& sp = B->plans[i]->steps[s];
        if (!sp.nftiles && !sp.skipA) pa.push_back({(int)i, &sp.copyA});
        if (!sp.skipB) pb.push_back({(int)i, &sp.copyB});
      }
      bs.A = merge_tasks(*B, pa);
      bs.B = merge_tasks(*B, pb);
      std::vector<GemmGroup> gg;
      std::vector<GemmTile> tt, ts;
      std::vector<SliceJob> jobs;
      std::vector<KexpJob> kjobs;
      std::vector<SplitGroup> sg;
      std::vector<GemmTile> st;
      std::vector<FusedTile> ft;
      std::vector<FusedCol> fc;
      for (size_t i = 0; i < B->plans.size(); ++i) {
        const StepPlan& sp = B->plans[i]->steps[s];
        const int b = B->base[i];
        const int goff = (int)gg.size();
        if (sp.nftiles) {
          // descriptors hold device addresses of the instance's own buffers;
          // tiles index the merged groups and descriptors
          const int coff = (int)fc.size();
          fc.insert(fc.end(), sp.hFC.begin(), sp.hFC.end());
          for (FusedTile t : sp.hFT) {
            t.group += goff;
            t.gcol += coff;
            if (t.scol >= 0) t.scol += coff;
            ft.push_back(t);
          }
          bs.fkp = std::max(bs.fkp, sp.fkp);
          bs.fnp = std::max(bs.fnp, sp.fnp);
        }
        for (GemmGroup g : sp.hG) {
          g.a_slot = shift_slot(g.a_slot, b);
          g.b_slot = shift_slot(g.b_slot, b);
          g.c_slot = shift_slot(g.c_slot, b);
          gg.push_back(g);
        }
        for (GemmTile t : sp.hT) { t.group += goff; tt.push_back(t); }
        if (!sp.nftiles)   // a fused instance's skinny tiles run inside its fused tiles
          for (GemmTile t : sp.hTs) { t.group += goff; ts.push_back(t); }
        bs.flops += sp.flops;
        bs.flops_skinny += sp.flops_skinny;
        if (split) {
          const int soff = (int)sg.size();
          for (size_t q = 0; q < sp.jobsAll.h.size(); ++q) {
            SliceJob j = sp.jobsAll.h[q];
            j.src_slot = shift_slot(j.src_slot, b);
            j.dst_slot = shift_slot(j.dst_slot, b);
            j.exp_slot = shift_slot(j.exp_slot, b);
            j.kx_slot = shift_slot(j.kx_slot, b);
            jobs.push_back(j);
          }
          for (KexpJob k : sp.hKJ) {
            k.src_slot = shift_slot(k.src_slot, b);
            k.kx_slot = shift_slot(k.kx_slot, b);
            kjobs.push_back(k);
          }
          bs.jobs.elems += sp.jobsAll.elems;
          for (SplitGroup g : sp.hSG) {
            g.a_slot = shift_slot(g.a_slot, b);
            g.b_slot = shift_slot(g.b_slot, b);
            g.c_slot = shift_slot(g.c_slot, b);
            g.ea_slot = shift_slot(g.ea_slot, b);
            g.eb_slot = shift_slot(g.eb_slot, b);
            sg.push_back(g);
          }
          for (GemmTile t : sp.hST) { t.group += soff; st.push_back(t); }
        }
      }
      bs.dG = B->upload(gg);
      bs.dT = B->upload(tt);
      bs.nt = (int)tt.size();
      bs.dTs = B->upload(ts);
      bs.nts = (int)ts.size();
      if (!ft.empty()) {
        if (ft.size() > (size_t)INT32_MAX) fail(TNX_ERR_UNSUPPORTED, "too many fused tiles in one batch");
        bs.dFT = B->upload(ft);
        bs.dFC = B->upload(fc);
        bs.nft = (int)ft.size();
      }
      if (split) {
        // longest K first, so a persistent grid ends with short tiles
        std::stable_sort(st.begin(), st.end(), [&](const GemmTile& x, const GemmTile& y) {
          return sg[x.group].K > sg[y.group].K;
        });
        // the merged launch is larger than any instance's: schedule it afresh
        const std::vector<int2> items =
            B->prec == TNX_PREC_TF32 ? tnx_tf32_schedule(jobs) : tnx_slice_schedule(jobs);
        bs.jobs.n = (int)jobs.size();
        bs.jobs.nitems = (int64_t)items.size();
        bs.jobs.d = B->upload(jobs);
        bs.jobs.items = B->upload(items);
        const std::vector<int4> kitems = tnx_kexp_items(kjobs);
        bs.dKJ = B->upload(kjobs);
        bs.nkj = (int)kjobs.size();
        bs.dKI = B->upload(kitems);
        bs.nki = (int64_t)kitems.size();
        bs.dSG = B->upload(sg);
        bs.dST = B->upload(st);
        bs.nst = (int)st.size();
        for (const GemmTile& t : st) bs.kmax = std::max(bs.kmax, (int)sg[t.group].K);
      }
    }
    std::vector<std::pair<int, const TaskList*>> pf;
    for (size_t i = 0; i < B->plans.size(); ++i) pf.push_back({(int)i, &B->plans[i]->fin});
    B->fin = merge_tasks(*B, pf);
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    *out = B.release();
  });
}

extern "C" tnx_status tnx_batch_destroy(tnx_batch* b) {
  if (!b) return TNX_ERR_ARG;
  cudaStreamSynchronize(b->ctx->stream);
  delete b;
  return TNX_OK;
}

extern "C" tnx_status tnx_batch_flops(tnx_batch* b, double* flops) {
  if (!b || !flops) return TNX_ERR_ARG;
  double f = 0;
  for (auto& s : b->steps) f += s.flops;
  *flops = f;
  return TNX_OK;
}

extern "C" tnx_status tnx_batch_launch_into(tnx_batch* b, tnx_tensor* const* outs) {
  if (!b) return TNX_ERR_ARG;
  return tnx_guard(b->ctx, [&] {
    if (!outs) fail(TNX_ERR_ARG, "null outputs");
    for (size_t i = 0; i < b->nets.size(); ++i)
      if (!outs[i]) fail(TNX_ERR_ARG, "null output tensor");
    check_fresh(*b);
    bind(*b, outs);
    tnx_ctx* c = b->ctx;
    if (c->stream && c->use_graphs) {
      if (!b->graph || b->graph->prof != c->prof) {
        b->graph.reset(new GraphRec());
        tnx_capture_graph(c, c->stream, *b->graph, [&] { enqueue_batch(*b, c->stream); });
      }
      CUDA_CHECK(cudaGraphLaunch(b->graph->exec, c->stream));
      tnx_note_launch(b->graph->nlaunch);
      if (c->prof) {
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        prof_accumulate(c, b->graph->recs);
      }
    } else {
      enqueue_batch(*b, c->stream);
    }
  });
}

extern "C" tnx_status tnx_batch_autotune(tnx_batch* b, tnx_tensor* const* outs, int* choice) {
  if (!b) return TNX_ERR_ARG;
  return tnx_guard(b->ctx, [&] {
    if (!outs) fail(TNX_ERR_ARG, "null outputs");
    check_fresh(*b);
    bind(*b, outs);
    tnx_ctx* c = b->ctx;
    const uint32_t prof = c->prof;
    c->prof = 0;
    const int cands[] = {0, 152, 304, 456};
    float best = 1e30f;
    int pick = 0;
    cudaEvent_t e0, e1;
    CUDA_CHECK(cudaEventCreate(&e0));
    CUDA_CHECK(cudaEventCreate(&e1));
    for (int cand : cands) {
      b->split_grid = cand;
      enqueue_batch(*b, c->stream);   // warm
      float t = 1e30f;
      for (int r = 0; r < 3; ++r) {
        CUDA_CHECK(cudaEventRecord(e0, c->stream));
        enqueue_batch(*b, c->stream);
        CUDA_CHECK(cudaEventRecord(e1, c->stream));
        CUDA_CHECK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
        t = std::min(t, ms);
      }
      if (t < best) {
        best = t;
        pick = cand;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->prof = prof;
    b->split_grid = pick;
    b->graph.reset();
    if (choice) *choice = pick;
  });
}
