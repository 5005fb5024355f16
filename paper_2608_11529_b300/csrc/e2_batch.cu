// C ABI: batches of planned problems evaluated with one persistent launch
// for their dense classes.
#include "e2_host.h"

#include <new>

using namespace e2;

extern "C" {

e2_status e2_batch_create(e2_problem* const* jobs, int n_jobs, e2_batch** out) {
  if (!out) return E2_ERR_INVALID_ARG;
  *out = nullptr;
  if (!jobs || n_jobs < 1) return E2_ERR_INVALID_ARG;
  e2_batch* B = new (std::nothrow) e2_batch();
  if (!B) return E2_ERR_OOM;
  Layout ws;
  int64_t njc = 0;
  for (int j = 0; j < n_jobs; ++j) {
    if (!jobs[j]) {
      delete B;
      return E2_ERR_INVALID_ARG;
    }
    B->jobs.push_back(jobs[j]);
    B->off.push_back(ws.take(jobs[j]->ws_bytes + (size_t)(jobs[j]->d.n_roots - 1) * jobs[j]->d_stride));
    for (int c : {2, 5, 7, 4, 6})
      if (jobs[j]->part_cnt[c] > 0 && !jobs[j]->use_oz[c]) {  // sliced classes launch on their own
        njc += jobs[j]->d.n_roots;
        B->n_items += jobs[j]->part_cnt[c] * jobs[j]->d.n_roots;
      }
  }
  if (B->n_items >= (int64_t)1 << 31) {
    delete B;
    return E2_ERR_UNSUPPORTED;
  }
  B->o_jobs = ws.take(sizeof(GemmJob) * std::max<int64_t>(njc, 1));
  B->o_items = ws.take(sizeof(WorkItem) * std::max<int64_t>(B->n_items, 1));
  B->o_counter = ws.take(sizeof(int));
  B->bytes = ws.top;
  *out = B;
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
  B->items.clear();
  struct Slots {  // every root of every job keeps its own tables for the batch's one launch
    e2_batch* b;
    explicit Slots(e2_batch* b_) : b(b_) { for (e2_problem* P : b->jobs) P->multi_slot = true; }
    ~Slots() { for (e2_problem* P : b->jobs) P->multi_slot = false; }
  } slots(B);
  struct Key {
    int kp;
    int job;
  };
  std::vector<Key> order;
  for (size_t j = 0; j < B->jobs.size(); ++j) {
    e2_problem* P = B->jobs[j];
    unsigned char* w = ws + B->off[j];
    for (int c : {2, 5, 7, 4, 6}) {
      if (P->part_cnt[c] == 0 || P->use_oz[c]) continue;
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
        // longest contraction first: the mean compacted length for a column-tiled class
        const int keff = P->use_cols[c] ? (int)(P->cplan[c].ratio * g.Kp + 0.5) : g.Kp;
        order.push_back({keff, (int)B->gj.size()});
        B->gj.push_back(g);
      }
    }
    if (cudaMemcpyAsync(w + P->o_plan, P->plan_blob.data(), P->plan_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return E2_ERR_CUDA;
  }
  // longest first: contraction length, then job order
  std::stable_sort(order.begin(), order.end(), [](const Key& x, const Key& y) { return x.kp > y.kp; });
  for (const Key& k : order) {
    const GemmJob& g = B->gj[k.job];
    const int ntm = (int)((g.M + 63) / 64), ntn = (int)((g.N + 63) / 64);
    for (int tm = 0; tm < ntm; ++tm)
      for (int tn = 0; tn < ntn; ++tn) B->items.push_back({k.job, tm, tn});
  }
  if ((int64_t)B->items.size() != B->n_items) return E2_ERR_SHAPE;
  if (cudaMemcpyAsync(ws + B->o_jobs, B->gj.data(), sizeof(GemmJob) * B->gj.size(), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(ws + B->o_items, B->items.data(), sizeof(WorkItem) * B->items.size(), cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
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
  struct Slots {
    e2_batch* b;
    explicit Slots(e2_batch* b_) : b(b_) { for (e2_problem* P : b->jobs) P->multi_slot = true; }
    ~Slots() { for (e2_problem* P : b->jobs) P->multi_slot = false; }
  } slots(B);
  for (size_t j = 0; j < B->jobs.size(); ++j) {
    e2_problem* P = B->jobs[j];
    unsigned char* w = ws + B->off[j];
    setup_common(P, inputs + j, w, st, false);
    setup_classes(P, w, st);
    for (int r = 0; r < P->d.n_roots; ++r)
      prepare_root(P, w, st, (const double2*)inputs[j].c + (int64_t)r * P->lists[P->listP].n, r);
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaMemsetAsync(ws + B->o_counter, 0, sizeof(int), st);
  if (B->n_items > 0)
    (k_batch_gemm<<<std::max(sms, 1), 256, 0, st>>>((const GemmJob*)(ws + B->o_jobs), (const WorkItem*)(ws + B->o_items),
                                                     (int)B->n_items, (int*)(ws + B->o_counter)), ++g_launches);
  auto nomark = [](int, int) {};
  for (size_t j = 0; j < B->jobs.size(); ++j) {
    e2_problem* P = B->jobs[j];
    unsigned char* w = ws + B->off[j];
    for (int c : {2, 5, 7, 6})
      if (P->use_oz[c] && P->part_cnt[c] > 0)
        for (int r = 0; r < P->d.n_roots; ++r)
          launch_class_oz(st, c, oz_operands(P, w, r, c), P->M[c], P->lists[P->list_of[c]].n,
                          (const RowInfo*)(w + P->o_rows[c]), (const double*)(w + P->o_E0p) + r,
                          P->d.level_shift_b, (double*)(w + P->o_part) + P->part_off[r * E2_NCLASS + c],
                          dmin_slot(P, w, r, c));
    for (int r = 0; r < P->d.n_roots; ++r)
      launch_sparse_classes(P, w, st, r, (const double2*)inputs[j].c + (int64_t)r * P->lists[P->listP].n, nomark);
    launch_reduce(P, w, st, E2[j], E2_class ? E2_class[j] : nullptr, nullptr);
  }
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
