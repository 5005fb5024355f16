// C ABI: batches of planned problems whose classes (every job, root and
// class) are evaluated by one persistent launch.
#include "e2_host.h"

#include <new>

using namespace e2;

extern "C" {

namespace {
// roots of job P that share one table slot group: all of them, or the batch's limit
int job_slots(const e2_batch* B, const e2_problem* P) {
  return B->roots_per_launch > 0 ? std::min(B->roots_per_launch, P->d.n_roots) : P->d.n_roots;
}

// Workspace of a batch: per job its forward layout with one table slot per
// root of a launch group and a copy of its coefficients, then the job lists,
// the runs and one work counter per launch.
void batch_layout(e2_batch* B) {
  Layout ws;
  B->off.clear();
  B->o_c.clear();
  B->max_gj = B->max_sj = 0;
  int max_roots = 1;
  for (const e2_problem* P : B->jobs) {
    B->off.push_back(ws.take(P->ws_bytes + (size_t)(job_slots(B, P) - 1) * P->d_stride));
    B->o_c.push_back(ws.take(16 * (size_t)P->lists[P->listP].n * P->d.n_roots));
    // at most one run per dense class and root, four per root for the element-wise classes
    B->max_gj += 5 * (int64_t)P->d.n_roots;
    B->max_sj += P->d.n_roots;
    max_roots = std::max(max_roots, P->d.n_roots);
  }
  B->n_launch = B->roots_per_launch > 0 ? (max_roots + B->roots_per_launch - 1) / B->roots_per_launch : 1;
  B->max_segs = B->max_gj + 4 * B->max_sj;
  B->o_jobs = ws.take(sizeof(GemmJob) * B->max_gj);
  B->o_sjobs = ws.take(sizeof(SparseJob) * B->max_sj);
  B->o_segs = ws.take(sizeof(WorkSeg) * B->max_segs);
  B->o_counter = ws.take(sizeof(unsigned long long) * B->n_launch);
  B->bytes = ws.top;
  B->prepared = nullptr;
}

// RAII: the batch's table slots are in use while a call runs
struct Slots {
  e2_batch* b;
  explicit Slots(e2_batch* b_) : b(b_) {
    for (e2_problem* P : b->jobs) {
      P->multi_slot = true;
      P->slots = job_slots(b, P);
    }
  }
  ~Slots() {
    for (e2_problem* P : b->jobs) {
      P->multi_slot = false;
      P->slots = 0;
    }
  }
};
}  // namespace

e2_status e2_batch_create(e2_problem* const* jobs, int n_jobs, e2_batch** out) {
  if (!out) return E2_ERR_INVALID_ARG;
  *out = nullptr;
  if (!jobs || n_jobs < 1) return E2_ERR_INVALID_ARG;
  e2_batch* B = new (std::nothrow) e2_batch();
  if (!B) return E2_ERR_OOM;
  for (int j = 0; j < n_jobs; ++j) {
    if (!jobs[j]) {
      delete B;
      return E2_ERR_INVALID_ARG;
    }
    B->jobs.push_back(jobs[j]);
  }
  batch_layout(B);
  *out = B;
  return E2_OK;
}

e2_status e2_batch_set_roots_per_launch(e2_batch* B, int k) {
  if (!B || k < 0) return E2_ERR_INVALID_ARG;
  B->roots_per_launch = k;
  batch_layout(B);
  return E2_OK;
}

e2_status e2_batch_destroy(e2_batch* B) {
  delete B;
  return E2_OK;
}

e2_status e2_batch_workspace_size(const e2_batch* B, size_t* bytes) {
  if (!B || !bytes) return E2_ERR_INVALID_ARG;
  *bytes = B->bytes;
  return E2_OK;
}

e2_status e2_batch_prepare(e2_batch* B, void* workspace, size_t workspace_bytes, void* stream_) {
  if (!B) return E2_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < B->bytes || ((uintptr_t)workspace & 255)) return E2_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream_;
  unsigned char* ws = (unsigned char*)workspace;
  B->gj.clear();
  B->sj.clear();
  B->segs.clear();
  B->seg0.clear();
  B->nseg.clear();
  B->items.clear();
  Slots slots(B);
  // a run of items, its launch (root group) and the FP64 work of one of its items (ordering key)
  struct Run {
    WorkSeg s;
    int launch;
    double cost;
  };
  std::vector<Run> runs;
  const int rpl = B->roots_per_launch;
  auto group = [rpl](int r) { return rpl > 0 ? r / rpl : 0; };
  for (size_t j = 0; j < B->jobs.size(); ++j) {
    e2_problem* P = B->jobs[j];
    unsigned char* w = ws + B->off[j];
    const int na = P->na;
    for (int c : {2, 5, 7, 4, 6}) {
      if (P->part_cnt[c] == 0 || P->use_oz[c]) continue;  // sliced classes launch on their own
      const DevList L = dev_list(P, P->list_of[c], w);
      for (int r = 0; r < P->d.n_roots; ++r) {
        Tabs T = tables(P, w, r);
        const double2* Dfor[E2_NCLASS] = {nullptr, nullptr, T.DTU, nullptr, T.DTDU, T.DT, T.DTDUD, T.DTD, nullptr};
        GemmJob g;
        g.W = (const double2*)(w + P->o_W[c]);
        g.D = Dfor[c];
        g.M = P->M[c];
        g.N = L.n;
        g.Kp = P->Kp[c];
        g.rows = (const RowInfo*)(w + P->o_rows[c]);
        g.U = L.U;
        g.eA = L.eA;
        g.E0p = (const double*)(w + P->o_E0p) + r;
        g.b = P->d.level_shift_b;
        g.partial = (double*)(w + P->o_part) + P->part_off[r * E2_NCLASS + c];
        g.ct = col_tiles(P, w, r, c);
        g.dmin = dmin_slot(P, w, r, c);
        // the mean compacted length for a column-tiled class
        const double keff = P->use_cols[c] ? P->cplan[c].ratio * g.Kp : g.Kp;
        const int64_t ntm = (g.M + 63) / 64, ntn = (g.N + 63) / 64;
        runs.push_back({WorkSeg{WORK_TILE, (int)B->gj.size(), 0, ntm * ntn, ntn}, group(r),
                        4096.0 * (3.0 * keff + 15.0)});
        B->gj.push_back(g);
      }
    }
    const Ctx X = ctx(P, w);
    for (int r = 0; r < P->d.n_roots; ++r) {
      const Tabs T = tables(P, w, r);
      SparseJob q{};
      q.L8 = dev_list(P, P->list_of[8], w);
      q.L1 = dev_list(P, P->list_of[1], w);
      q.L3 = dev_list(P, P->list_of[3], w);
      q.L0 = dev_list(P, P->list_of[0], w);
      q.L2 = dev_list(P, P->list_of[2], w);
      q.L4 = dev_list(P, P->list_of[4], w);
      q.L5 = dev_list(P, P->list_of[5], w);
      q.L7 = dev_list(P, P->list_of[7], w);
      q.das = P->das;
      q.sp = X.sp;
      q.binom = X.binom;
      q.c = (const double2*)(ws + B->o_c[j]) + (int64_t)r * P->lists[P->listP].n;
      q.DT = T.DT;
      q.DTU = T.DTU;
      q.DTD = T.DTD;
      q.DTDU = T.DTDU;
      q.X01 = (const double2*)(w + P->o_X01);
      q.X10 = (const double2*)(w + P->o_X10);
      q.X00 = (const double2*)(w + P->o_X00);
      q.f = X.f;
      q.g2 = (const double*)(w + P->o_G22);
      q.epsh = X.epsh;
      q.G = X.G;
      q.E0p = X.E0p + r;
      q.b = P->d.level_shift_b;
      q.nvb = P->nvb;
      const int cls4[4] = {8, 1, 3, 0};
      for (int k = 0; k < 4; ++k) {
        q.part[k] = (double*)(w + P->o_part) + P->part_off[r * E2_NCLASS + cls4[k]];
        q.dmin[k] = dmin_slot(P, w, r, cls4[k]);
      }
      const int sjob = (int)B->sj.size();
      bool any = false;
      if (shard_units(P, 8) > 0 && !P->use_oz[8]) {  // the float-float (2,2) launches on its own
        const int64_t gx = blocks(q.L8.n);
        runs.push_back({WorkSeg{WORK_C22, sjob, 0, shard_units(P, 8) * gx, gx}, group(r), 256.0 * 64 * 8});
        any = true;
      }
      if (shard_units(P, 1) > 0) {
        const int64_t gx = blocks(q.L1.n), cnt = q.L1.count;
        runs.push_back({WorkSeg{WORK_C01, sjob, 0, shard_units(P, 1) * gx, gx}, group(r),
                        256.0 * 4 * (na + cnt * (double)(na - cnt + 1) * (na - cnt) / 2)});
        any = true;
      }
      if (shard_units(P, 3) > 0) {
        const int64_t gx = blocks(q.L3.n), cnt = q.L3.count;
        runs.push_back({WorkSeg{WORK_C10, sjob, 0, shard_units(P, 3) * gx, gx}, group(r),
                        256.0 * 4 * (na + (double)cnt * (cnt - 1) / 2 * (na - cnt + 2))});
        any = true;
      }
      if (shard_units(P, 0) > 0) {
        const int64_t cnt = q.L0.count;
        runs.push_back({WorkSeg{WORK_C00, sjob, 0, shard_units(P, 0), 1}, group(r),
                        256.0 * 4 * (cnt * (double)(na - cnt) + (double)cnt * (cnt - 1) / 2 * (na - cnt) *
                                                                     (na - cnt - 1) / 2)});
        any = true;
      }
      if (any) B->sj.push_back(q);
    }
    if (cudaMemcpyAsync(w + P->o_plan, P->plan_blob.data(), P->plan_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return E2_ERR_CUDA;
  }
  if ((int64_t)B->gj.size() > B->max_gj || (int64_t)B->sj.size() > B->max_sj ||
      (int64_t)runs.size() > B->max_segs)
    return E2_ERR_SHAPE;
  // per launch, longest item first (FP64 operations per item), then job order
  std::stable_sort(runs.begin(), runs.end(), [](const Run& x, const Run& y) {
    return x.launch != y.launch ? x.launch < y.launch : x.cost > y.cost;
  });
  B->n_items = 0;
  size_t i = 0;
  for (int g = 0; g < B->n_launch; ++g) {
    B->seg0.push_back((int64_t)B->segs.size());
    int64_t first = 0;  // items are numbered within their launch
    for (; i < runs.size() && runs[i].launch == g; ++i) {
      runs[i].s.first = first;
      first += runs[i].s.count;
      B->segs.push_back(runs[i].s);
    }
    B->nseg.push_back((int64_t)B->segs.size() - B->seg0.back());
    B->items.push_back(first);
    B->n_items += first;
  }
  if ((!B->gj.empty() && cudaMemcpyAsync(ws + B->o_jobs, B->gj.data(), sizeof(GemmJob) * B->gj.size(),
                                         cudaMemcpyHostToDevice, st) != cudaSuccess) ||
      (!B->sj.empty() && cudaMemcpyAsync(ws + B->o_sjobs, B->sj.data(), sizeof(SparseJob) * B->sj.size(),
                                         cudaMemcpyHostToDevice, st) != cudaSuccess) ||
      (!B->segs.empty() && cudaMemcpyAsync(ws + B->o_segs, B->segs.data(), sizeof(WorkSeg) * B->segs.size(),
                                           cudaMemcpyHostToDevice, st) != cudaSuccess))
    return E2_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return E2_ERR_CUDA;
  B->prepared = workspace;
  return E2_OK;
}

e2_status e2_batch_forward(e2_batch* B, const e2_inputs* inputs, void* workspace, size_t workspace_bytes,
                           void* stream_, double* const* E2, double* const* E2_class) {
  if (!B || !inputs || !E2) return E2_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < B->bytes || workspace != B->prepared) return E2_ERR_WORKSPACE;
  for (size_t j = 0; j < B->jobs.size(); ++j) {
    if (B->jobs[j]->shard_n > 1) return E2_ERR_UNSUPPORTED;  // batches run unsharded
    const e2_inputs* in = inputs + j;
    if (!E2[j] || !in->h || !in->B_c || !in->c || !std::isfinite(in->lambda)) return E2_ERR_INVALID_ARG;
    if (B->jobs[j]->d.L_extra > 0 && (!in->B_x || !in->w_x)) return E2_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream_;
  unsigned char* ws = (unsigned char*)workspace;
  cudaGetLastError();
  g_launches = 0;
  Slots slots(B);
  for (size_t j = 0; j < B->jobs.size(); ++j) {
    e2_problem* P = B->jobs[j];
    unsigned char* w = ws + B->off[j];
    setup_common(P, inputs + j, w, st, false);
    setup_classes(P, w, st);
    // the element-wise classes read c from the batch's own copy (device to device)
    if (cudaMemcpyAsync(ws + B->o_c[j], inputs[j].c, 16 * (size_t)P->lists[P->listP].n * P->d.n_roots,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return E2_ERR_CUDA;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int rpl = B->roots_per_launch;
  for (int g = 0; g < B->n_launch; ++g) {
    // the roots of this launch: their coupling tables in the jobs' slots
    auto in_group = [&](int r) { return rpl > 0 ? r / rpl == g : true; };
    for (size_t j = 0; j < B->jobs.size(); ++j) {
      e2_problem* P = B->jobs[j];
      unsigned char* w = ws + B->off[j];
      const int64_t np = P->lists[P->listP].n;
      for (int r = 0; r < P->d.n_roots; ++r)
        if (in_group(r)) prepare_root(P, w, st, (const double2*)inputs[j].c + (int64_t)r * np, r);
    }
    unsigned long long* counter = (unsigned long long*)(ws + B->o_counter) + g;
    cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
    if (B->items[g] > 0)
      (k_batch<<<std::max(sms, 1), 256, 0, st>>>((const WorkSeg*)(ws + B->o_segs) + B->seg0[g], (int)B->nseg[g],
                                                  (const GemmJob*)(ws + B->o_jobs),
                                                  (const SparseJob*)(ws + B->o_sjobs), B->items[g], counter),
       ++g_launches);
    for (size_t j = 0; j < B->jobs.size(); ++j) {  // classes a job opted into the emulated arithmetic
      e2_problem* P = B->jobs[j];
      unsigned char* w = ws + B->off[j];
      const DevList L8 = dev_list(P, P->list_of[8], w);
      const Ctx X = ctx(P, w);
      for (int r = 0; r < P->d.n_roots; ++r) {
        if (!in_group(r)) continue;
        for (int c : {2, 5, 7, 6})
          if (P->use_oz[c] && P->part_cnt[c] > 0)
            launch_class_oz(st, c, oz_operands(P, w, r, c), P->M[c], P->lists[P->list_of[c]].n,
                            (const RowInfo*)(w + P->o_rows[c]), (const double*)(w + P->o_E0p) + r,
                            P->d.level_shift_b, (double*)(w + P->o_part) + P->part_off[r * E2_NCLASS + c],
                            dmin_slot(P, w, r, c));
        if (P->use_oz[8] && shard_units(P, 8) > 0) {
          const HostList& H8 = P->lists[P->list_of[8]];
          launch_class22_df(st, L8, X.sp, (const float2*)(w + H8.o_eAdf), (const float2*)(w + H8.o_Udf),
                            (const double2*)inputs[j].c + (int64_t)r * P->lists[P->listP].n,
                            (const double*)(w + P->o_G22), X.epsh, X.G, X.E0p + r, P->d.level_shift_b, P->nvb,
                            P->ncp, (double*)(w + P->o_part) + P->part_off[r * E2_NCLASS + 8],
                            dmin_slot(P, w, r, 8));
        }
      }
    }
  }
  for (size_t j = 0; j < B->jobs.size(); ++j)
    launch_reduce(B->jobs[j], ws + B->off[j], st, E2[j], E2_class ? E2_class[j] : nullptr, nullptr);
  B->launches = g_launches;
  if (cudaGetLastError() != cudaSuccess) return E2_ERR_CUDA;
  return E2_OK;
}

e2_status e2_batch_backward_workspace_size(const e2_batch* B, size_t* bytes) {
  if (!B || !bytes) return E2_ERR_INVALID_ARG;
  size_t m = 0;
  for (const e2_problem* P : B->jobs) m = std::max(m, P->bwd_bytes);
  *bytes = m;
  return E2_OK;
}

e2_status e2_batch_backward(e2_batch* B, const e2_inputs* inputs, const double* const* seeds, void* workspace,
                            size_t workspace_bytes, void* stream, double* const* g_h, double* const* g_c,
                            double* const* g_Bc, double* const* g_Bx, double* const* dE2_dlambda,
                            double* const* E2) {
  if (!B || !inputs || !seeds) return E2_ERR_INVALID_ARG;
  size_t need = 0;
  e2_batch_backward_workspace_size(B, &need);
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255)) return E2_ERR_WORKSPACE;
  for (size_t j = 0; j < B->jobs.size(); ++j)
    if (!seeds[j]) return E2_ERR_INVALID_ARG;
  auto at = [](double* const* a, size_t j) { return a ? a[j] : nullptr; };
  int64_t launches = 0;
  for (size_t j = 0; j < B->jobs.size(); ++j) {
    const e2_status st = e2_backward(B->jobs[j], inputs + j, seeds[j], workspace, workspace_bytes, stream,
                                     at(g_h, j), at(g_c, j), at(g_Bc, j), at(g_Bx, j), at(dE2_dlambda, j), at(E2, j));
    if (st != E2_OK) return st;
    launches += B->jobs[j]->launches;
  }
  B->launches = launches;
  return E2_OK;
}

e2_status e2_batch_launch_count(const e2_batch* B, int64_t* n) {
  if (!B || !n) return E2_ERR_INVALID_ARG;
  *n = B->launches;
  return E2_OK;
}

}  // extern "C"
