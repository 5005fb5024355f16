// C ABI: host plan (occupation patterns, string lists, workspace layout) and
// the stream-ordered launch sequence of e2_forward.  No device allocation.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "e2_common.cuh"
#include "e2_kernels.cuh"

using namespace e2;

namespace {

using Pat = std::array<int, E2_MAX_DAS>;

int64_t binom_h(int n, int k) {
  if (k < 0 || n < 0 || k > n) return 0;
  int64_t r = 1;
  int kk = std::min(k, n - k);
  for (int j = 1; j <= kk; ++j) r = r * (n - kk + j) / j;
  return r;
}

struct HostList {
  int count = 0;
  std::vector<Pat> pats;
  std::vector<int64_t> patoff;
  int64_t n = 0;
  std::vector<int64_t> key2off;
  size_t o_str = 0, o_key = 0, o_patoff = 0, o_patocc = 0, o_eA = 0, o_U = 0;
};

// Bump allocator over the workspace (256-byte aligned segments).
struct Layout {
  size_t top = 0;
  size_t take(size_t bytes) {
    size_t o = top;
    top += (bytes + 255) & ~size_t(255);
    return o;
  }
};

}  // namespace

struct e2_problem {
  e2_desc d;
  std::vector<uint8_t> frozen;
  int das_size[E2_MAX_DAS], das_min[E2_MAX_DAS], das_max[E2_MAX_DAS];
  int n, nocc, ncc, nvc, nx, na, N;
  std::vector<int32_t> cc, vc;
  DevDas das;
  int nkeys;
  std::vector<Pat> ppats;          // P patterns (address order)
  std::vector<HostList> lists;     // unique string lists
  int list_of[E2_NCLASS];          // class -> list (-1: no strings)
  int listP;
  // integral / table shapes
  int ntp;
  int64_t nvp, ncp;
  int64_t M[E2_NCLASS];            // rows of each class
  int Kp[E2_NCLASS];               // padded contraction length of the dense classes
  int KpT, KpTU, Kp11;             // rows of the D^t / D^tu / D^{t+u} tables
  double q_per_class[E2_NCLASS];
  // workspace layout
  size_t ws_bytes;
  size_t o_plan, plan_bytes;
  size_t o_binom, o_EO, o_E0p, o_E0, o_G, o_epsh, o_dg, o_wt, o_Bo, o_f, o_cc, o_vc;
  size_t o_rows[E2_NCLASS], o_W[E2_NCLASS];
  size_t o_G22, o_X01, o_X10, o_X00;
  size_t o_DT, o_DTD, o_DTU, o_DTDUD, o_DTDU;  // per-root stride below
  size_t d_stride;                              // bytes per root of all D tables
  size_t o_g1, o_g2, g_stride;                  // gram outputs per root
  size_t o_part, o_partoff, o_partcnt, o_e2c;
  int64_t part_cnt[E2_NCLASS];
  std::vector<int64_t> part_off;                // [n_roots][E2_NCLASS]
  std::vector<unsigned char> plan_blob;         // host image of the plan region
  // launch shapes of the sparse / elementwise classes
  int nvb;
};

namespace {

bool pattern_allowed(const e2_problem* P, const Pat& pt) {
  for (int s = 0; s < P->d.n_das; ++s)
    if (pt[s] < P->das_min[s] || pt[s] > P->das_max[s]) return false;
  return true;
}

// all occupation patterns with `count` electrons, lexicographic (n_1 most significant)
std::vector<Pat> all_patterns(const e2_problem* P, int count) {
  std::vector<Pat> out;
  Pat cur{};
  struct Rec {
    static void go(const e2_problem* P, int s, int left, Pat& cur, std::vector<Pat>& out) {
      if (s == P->d.n_das) {
        if (left == 0) out.push_back(cur);
        return;
      }
      for (int k = 0; k <= P->das_size[s] && k <= left; ++k) {
        cur[s] = k;
        go(P, s + 1, left - k, cur, out);
      }
      cur[s] = 0;
    }
  };
  Rec::go(P, 0, count, cur, out);
  return out;
}

int min_deficit(const e2_problem* P, const Pat& pt) {
  int best = 1 << 30;
  for (const Pat& q : P->ppats) {
    int d = 0;
    for (int s = 0; s < P->d.n_das; ++s) d += std::max(0, q[s] - pt[s]);
    best = std::min(best, d);
  }
  return best;
}

int64_t pattern_size(const e2_problem* P, const Pat& pt) {
  int64_t c = 1;
  for (int s = 0; s < P->d.n_das; ++s) c *= binom_h(P->das_size[s], pt[s]);
  return c;
}

int key_of(const e2_problem* P, const Pat& pt) {
  int k = 0;
  for (int s = 0; s < P->d.n_das; ++s) k += pt[s] * P->das.keymul[s];
  return k;
}

int add_list(e2_problem* P, int count, const std::vector<Pat>& pats) {
  for (size_t i = 0; i < P->lists.size(); ++i)
    if (P->lists[i].count == count && P->lists[i].pats == pats) return (int)i;
  HostList L;
  L.count = count;
  L.pats = pats;
  L.key2off.assign(P->nkeys, -1);
  int64_t off = 0;
  for (const Pat& pt : pats) {
    L.patoff.push_back(off);
    L.key2off[key_of(P, pt)] = off;
    off += pattern_size(P, pt);
  }
  L.n = off;
  P->lists.push_back(L);
  return (int)P->lists.size() - 1;
}

template <class T>
void put(std::vector<unsigned char>& blob, size_t off, const T* src, size_t count) {
  if (count) std::memcpy(blob.data() + off, src, sizeof(T) * count);
}

e2_status build_plan(e2_problem* P) {
  const e2_desc& d = P->d;
  P->na = d.n_active;
  P->N = d.n_elec;
  P->n = d.n_core + d.n_active + d.n_virt;
  P->nocc = d.n_core + d.n_active;
  for (int k = 0; k < d.n_core; ++k)
    if (!P->frozen[k]) P->cc.push_back(k);
  for (int v = P->nocc; v < P->n; ++v)
    if (!P->frozen[v]) P->vc.push_back(v);
  P->ncc = (int)P->cc.size();
  P->nvc = (int)P->vc.size();
  P->nx = P->ncc + P->nvc;
  P->ntp = (int)pairs(P->na);
  P->nvp = pairs(P->nvc);
  P->ncp = pairs(P->ncc);
  // partition
  P->das.n_das = d.n_das;
  P->das.n_act = d.n_active;
  int off = 0, mul = 1;
  for (int s = 0; s < d.n_das; ++s) {
    P->das.off[s] = off;
    P->das.size[s] = P->das_size[s];
    P->das.keymul[s] = mul;
    off += P->das_size[s];
    if ((int64_t)mul * (P->das_size[s] + 1) > kMaxKeys) return E2_ERR_UNSUPPORTED;
    mul *= P->das_size[s] + 1;
  }
  P->nkeys = mul;
  for (const Pat& pt : all_patterns(P, P->N))
    if (pattern_allowed(P, pt)) P->ppats.push_back(pt);
  if (P->ppats.empty()) return E2_ERR_SHAPE;
  P->listP = add_list(P, P->N, P->ppats);
  // class lists: strings of N+h-p electrons within two substitutions of P
  for (int h = 0; h <= 2; ++h)
    for (int p = 0; p <= 2; ++p) {
      const int cls = 3 * h + p, cnt = P->N + h - p;
      P->list_of[cls] = -1;
      if (cnt < 0 || cnt > P->na) continue;
      std::vector<Pat> pats;
      for (const Pat& pt : all_patterns(P, cnt)) {
        if (h + min_deficit(P, pt) > 2) continue;
        if (h == 0 && p == 0 && pattern_allowed(P, pt)) continue;
        pats.push_back(pt);
      }
      if ((int)pats.size() > kMaxPat) return E2_ERR_UNSUPPORTED;
      if (pats.empty()) continue;
      P->list_of[cls] = add_list(P, cnt, pats);
    }
  // class (2,2) strings carry no substitution: they are exactly P, and the
  // (2,2) kernel reads c by list position
  if (P->list_of[8] >= 0 && P->list_of[8] != P->listP) return E2_ERR_UNSUPPORTED;
  // rows per class
  const int64_t nc = P->ncc, nv = P->nvc;
  const int64_t rows[E2_NCLASS] = {1, nv, P->nvp, nc, nc * nv, nc * P->nvp, P->ncp, P->ncp * nv, P->ncp * P->nvp};
  for (int c = 0; c < E2_NCLASS; ++c) {
    P->M[c] = (P->list_of[c] >= 0) ? rows[c] : 0;
    P->q_per_class[c] = (P->list_of[c] >= 0) ? (double)rows[c] * (double)P->lists[P->list_of[c]].n : 0.0;
  }
  auto pad8 = [](int k) { return (k + 7) / 8 * 8; };
  P->KpT = pad8(P->na);
  P->KpTU = pad8(std::max(P->ntp, 1));
  P->Kp11 = pad8(1 + P->na * P->na);
  for (int c = 0; c < E2_NCLASS; ++c) P->Kp[c] = 0;
  P->Kp[2] = P->KpTU;
  P->Kp[5] = P->KpT;
  P->Kp[7] = P->KpT;
  P->Kp[4] = P->Kp11;
  P->Kp[6] = P->KpTU;

  // ---- workspace layout
  Layout ws;
  const int R = d.n_roots;
  const int Lt = d.L_coulomb + d.L_extra;
  // plan region first: everything the host computes, uploaded in one copy
  P->o_plan = ws.take(0);
  P->o_cc = ws.take(sizeof(int32_t) * std::max(1, P->ncc));
  P->o_vc = ws.take(sizeof(int32_t) * std::max(1, P->nvc));
  for (HostList& L : P->lists) {
    L.o_key = ws.take(sizeof(int64_t) * P->nkeys);
    L.o_patoff = ws.take(sizeof(int64_t) * L.pats.size());
    L.o_patocc = ws.take(sizeof(int32_t) * E2_MAX_DAS * L.pats.size());
  }
  P->o_partoff = ws.take(sizeof(int64_t) * R * E2_NCLASS);
  P->o_partcnt = ws.take(sizeof(int64_t) * E2_NCLASS);
  P->plan_bytes = ws.top - P->o_plan;
  // device-computed data
  P->o_binom = ws.take(sizeof(int64_t) * kBinomN * kBinomN);
  P->o_EO = ws.take(sizeof(double));
  P->o_E0p = ws.take(sizeof(double) * R);
  P->o_E0 = ws.take(sizeof(double) * R);
  P->o_G = ws.take(sizeof(double) * P->n * P->n);
  P->o_epsh = ws.take(sizeof(double) * P->n);
  P->o_dg = ws.take(sizeof(double) * Lt * P->n);
  P->o_wt = ws.take(sizeof(double) * Lt);
  P->o_Bo = ws.take(16 * (size_t)Lt * P->n * P->nocc);
  P->o_f = ws.take(16 * (size_t)P->n * P->nocc);
  for (HostList& L : P->lists) {
    L.o_str = ws.take(sizeof(uint64_t) * std::max<int64_t>(L.n, 1));
    L.o_eA = ws.take(sizeof(double) * std::max<int64_t>(L.n, 1));
    L.o_U = ws.take(sizeof(double) * (size_t)(P->nx + 1) * std::max<int64_t>(L.n, 1));
  }
  const int dense[5] = {2, 5, 7, 4, 6};
  for (int c = 0; c < E2_NCLASS; ++c) P->o_rows[c] = P->o_W[c] = 0;
  for (int c : dense) {
    if (P->M[c] == 0) continue;
    P->o_rows[c] = ws.take(sizeof(RowInfo) * P->M[c]);
    P->o_W[c] = ws.take(16 * (size_t)P->M[c] * P->Kp[c]);
  }
  P->o_G22 = ws.take(sizeof(double) * std::max<int64_t>(P->ncp * P->nvp, 1));
  P->o_X01 = ws.take(16 * (size_t)std::max<int64_t>((int64_t)P->nvc * P->na * P->ntp, 1));
  P->o_X10 = ws.take(16 * (size_t)std::max<int64_t>((int64_t)P->ncc * P->ntp * P->na, 1));
  P->o_X00 = ws.take(16 * (size_t)std::max<int64_t>((int64_t)P->ntp * P->ntp, 1));
  // D tables (per root)
  auto lsize = [&](int cls) -> int64_t { return P->list_of[cls] >= 0 ? P->lists[P->list_of[cls]].n : 0; };
  size_t dstart = ws.top;
  P->o_DT = ws.take(16 * (size_t)P->KpT * std::max<int64_t>(lsize(5), 1));
  P->o_DTD = ws.take(16 * (size_t)P->KpT * std::max<int64_t>(lsize(7), 1));
  P->o_DTU = ws.take(16 * (size_t)P->KpTU * std::max<int64_t>(lsize(2), 1));
  P->o_DTDUD = ws.take(16 * (size_t)P->KpTU * std::max<int64_t>(lsize(6), 1));
  P->o_DTDU = ws.take(16 * (size_t)P->Kp11 * std::max<int64_t>(lsize(4), 1));
  P->d_stride = ws.top - dstart;
  ws.top = dstart + P->d_stride * R;
  size_t gstart = ws.top;
  P->o_g1 = ws.take(16 * (size_t)(1 + P->na * P->na));
  P->o_g2 = ws.take(16 * (size_t)std::max(P->ntp * P->ntp, 1));
  P->g_stride = ws.top - gstart;
  ws.top = gstart + P->g_stride * R;
  // partials
  P->nvb = (P->nvc + 7) / 8;
  for (int c = 0; c < E2_NCLASS; ++c) {
    int64_t cnt = 0;
    const int li = P->list_of[c];
    const int64_t nA = li >= 0 ? P->lists[li].n : 0;
    const bool on = (d.class_mask >> c) & 1u;
    if (on && P->M[c] > 0 && nA > 0) {
      if (c == 2 || c == 5 || c == 7 || c == 4 || c == 6) cnt = ((P->M[c] + 63) / 64) * ((nA + 63) / 64);
      else if (c == 8) cnt = ((nA + 255) / 256) * ((int64_t)P->nvb * (P->nvb + 1) / 2) * P->ncp;
      else if (c == 1) cnt = ((nA + 255) / 256) * P->nvc;
      else if (c == 3) cnt = ((nA + 255) / 256) * P->ncc;
      else if (c == 0) cnt = (nA + 255) / 256;
    }
    P->part_cnt[c] = cnt;
  }
  int64_t tot = 0;
  P->part_off.assign((size_t)R * E2_NCLASS, 0);
  for (int r = 0; r < R; ++r)
    for (int c = 0; c < E2_NCLASS; ++c) {
      P->part_off[r * E2_NCLASS + c] = tot;
      tot += P->part_cnt[c];
    }
  P->o_part = ws.take(sizeof(double) * std::max<int64_t>(tot, 1));
  P->o_e2c = ws.take(sizeof(double) * R * E2_NCLASS);
  P->ws_bytes = ws.top;

  // ---- host image of the plan region
  P->plan_blob.assign(P->plan_bytes, 0);
  auto rel = [&](size_t o) { return o - P->o_plan; };
  put(P->plan_blob, rel(P->o_cc), P->cc.data(), P->cc.size());
  put(P->plan_blob, rel(P->o_vc), P->vc.data(), P->vc.size());
  for (HostList& L : P->lists) {
    put(P->plan_blob, rel(L.o_key), L.key2off.data(), L.key2off.size());
    put(P->plan_blob, rel(L.o_patoff), L.patoff.data(), L.patoff.size());
    std::vector<int32_t> occ(E2_MAX_DAS * L.pats.size(), 0);
    for (size_t k = 0; k < L.pats.size(); ++k)
      for (int s = 0; s < E2_MAX_DAS; ++s) occ[k * E2_MAX_DAS + s] = L.pats[k][s];
    put(P->plan_blob, rel(L.o_patocc), occ.data(), occ.size());
  }
  put(P->plan_blob, rel(P->o_partoff), P->part_off.data(), P->part_off.size());
  put(P->plan_blob, rel(P->o_partcnt), P->part_cnt, E2_NCLASS);
  return E2_OK;
}

DevList dev_list(const e2_problem* P, int li, unsigned char* ws) {
  DevList D{};
  if (li < 0) return D;
  const HostList& L = P->lists[li];
  D.count = L.count;
  D.npat = (int)L.pats.size();
  D.n = L.n;
  D.str = (uint64_t*)(ws + L.o_str);
  D.key2off = (const int64_t*)(ws + L.o_key);
  D.patoff = (const int64_t*)(ws + L.o_patoff);
  D.patocc = (const int32_t*)(ws + L.o_patocc);
  D.eA = (double*)(ws + L.o_eA);
  D.U = (double*)(ws + L.o_U);
  return D;
}

inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

extern "C" {

const char* e2_status_string(e2_status s) {
  switch (s) {
    case E2_OK: return "ok";
    case E2_ERR_INVALID_ARG: return "invalid argument";
    case E2_ERR_SHAPE: return "inconsistent shape or empty reference space";
    case E2_ERR_UNSUPPORTED: return "unsupported size";
    case E2_ERR_WORKSPACE: return "workspace too small or misaligned";
    case E2_ERR_CUDA: return "CUDA error";
    case E2_ERR_NONFINITE: return "non-finite value";
  }
  return "unknown status";
}

e2_status e2_problem_create(const e2_desc* desc, e2_problem** out) {
  if (!out) return E2_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc) return E2_ERR_INVALID_ARG;
  const e2_desc& d = *desc;
  if (d.n_core < 0 || d.n_virt < 0 || d.n_active < 1 || d.n_active > 62) return E2_ERR_SHAPE;
  if (d.n_elec < 0 || d.n_elec > d.n_active) return E2_ERR_SHAPE;
  if (d.n_das < 1 || d.n_das > E2_MAX_DAS || !d.das_size || !d.das_min || !d.das_max) return E2_ERR_INVALID_ARG;
  if (d.ham < E2_DC || d.ham > E2_DCB || d.L_coulomb < 1 || d.L_extra < 0) return E2_ERR_INVALID_ARG;
  if (d.ham == E2_DC && d.L_extra != 0) return E2_ERR_INVALID_ARG;
  if (d.n_roots < 1 || d.n_roots > 16) return E2_ERR_INVALID_ARG;
  if (!(d.level_shift_b >= 0.0) || !std::isfinite(d.level_shift_b)) return E2_ERR_INVALID_ARG;
  int sum = 0;
  for (int s = 0; s < d.n_das; ++s) {
    if (d.das_size[s] < 1 || d.das_min[s] < 0 || d.das_max[s] < d.das_min[s] || d.das_min[s] > d.das_size[s])
      return E2_ERR_SHAPE;
    sum += d.das_size[s];
  }
  if (sum != d.n_active) return E2_ERR_SHAPE;
  const int n = d.n_core + d.n_active + d.n_virt;
  e2_problem* P = new (std::nothrow) e2_problem();
  if (!P) return E2_ERR_INVALID_ARG;
  P->d = d;
  P->frozen.assign(n, 0);
  if (d.frozen) {
    for (int p = 0; p < n; ++p) P->frozen[p] = d.frozen[p] ? 1 : 0;
    for (int t = d.n_core; t < d.n_core + d.n_active; ++t)
      if (P->frozen[t]) {
        delete P;
        return E2_ERR_SHAPE;
      }
  }
  for (int s = 0; s < d.n_das; ++s) {
    P->das_size[s] = d.das_size[s];
    P->das_min[s] = d.das_min[s];
    P->das_max[s] = std::min(d.das_max[s], d.das_size[s]);
  }
  P->d.frozen = nullptr;
  P->d.das_size = P->das_size;
  P->d.das_min = P->das_min;
  P->d.das_max = P->das_max;
  e2_status st;
  try {
    st = build_plan(P);
  } catch (...) {
    st = E2_ERR_UNSUPPORTED;
  }
  if (st != E2_OK) {
    delete P;
    return st;
  }
  *out = P;
  return E2_OK;
}

e2_status e2_problem_destroy(e2_problem* prob) {
  delete prob;
  return E2_OK;
}

e2_status e2_problem_info(const e2_problem* P, int64_t* n_p, double* q_per_class) {
  if (!P) return E2_ERR_INVALID_ARG;
  if (n_p) *n_p = P->lists[P->listP].n;
  if (q_per_class)
    for (int c = 0; c < E2_NCLASS; ++c) q_per_class[c] = P->q_per_class[c];
  return E2_OK;
}

e2_status e2_workspace_size(const e2_problem* P, size_t* bytes) {
  if (!P || !bytes) return E2_ERR_INVALID_ARG;
  *bytes = P->ws_bytes;
  return E2_OK;
}

e2_status e2_forward(e2_problem* P, const e2_inputs* in, void* workspace, size_t workspace_bytes, void* stream_,
                     double* E2, double* E2_class, double* E0) {
  if (!P || !in || !E2 || !in->h || !in->B_c || !in->c) return E2_ERR_INVALID_ARG;
  if (P->d.L_extra > 0 && (!in->B_x || !in->w_x)) return E2_ERR_INVALID_ARG;
  if (!std::isfinite(in->lambda)) return E2_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < P->ws_bytes || ((uintptr_t)workspace & 255)) return E2_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream_;
  unsigned char* ws = (unsigned char*)workspace;
  const e2_desc& d = P->d;
  const int n = P->n, nocc = P->nocc, na = P->na, R = d.n_roots, Lt = d.L_coulomb + d.L_extra;
  const double b = d.level_shift_b;

  auto W = [&](size_t o) { return (void*)(ws + o); };
  const int64_t* binom = (const int64_t*)W(P->o_binom);
  double* G = (double*)W(P->o_G);
  double* epsh = (double*)W(P->o_epsh);
  double* EO = (double*)W(P->o_EO);
  double* E0p = (double*)W(P->o_E0p);
  double* E0d = (double*)W(P->o_E0);
  double* dg = (double*)W(P->o_dg);
  double* wt = (double*)W(P->o_wt);
  double2* Bo = (double2*)W(P->o_Bo);
  double2* f = (double2*)W(P->o_f);

  DevSpace sp;
  sp.n = n;
  sp.n_core = d.n_core;
  sp.n_act = na;
  sp.n_virt = d.n_virt;
  sp.n_occ = nocc;
  sp.a0 = d.n_core;
  sp.v0 = nocc;
  sp.ncc = P->ncc;
  sp.nvc = P->nvc;
  sp.nx = P->nx;
  sp.cc = (const int32_t*)W(P->o_cc);
  sp.vc = (const int32_t*)W(P->o_vc);

  cudaGetLastError();
  if (cudaMemcpyAsync(W(P->o_plan), P->plan_blob.data(), P->plan_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return E2_ERR_CUDA;
  k_binom<<<1, 256, 0, st>>>((int64_t*)W(P->o_binom));
  {
    int64_t tot = (int64_t)Lt * n * nocc;
    unsigned g = (unsigned)std::min<int64_t>(blocks(tot), 148 * 64);
    k_extract<<<g, 256, 0, st>>>((const double2*)in->B_c, (const double2*)in->B_x, in->w_x, in->lambda, d.L_coulomb,
                                 d.L_extra, n, nocc, Bo, wt, dg);
  }
  k_G<<<blocks((int64_t)n * n), 256, 0, st>>>((const double2*)in->B_c, (const double2*)in->B_x, wt, dg, d.L_coulomb,
                                              d.L_extra, n, G);
  k_fock<<<blocks((int64_t)n * nocc), 256, 0, st>>>((const double2*)in->h, Bo, wt, dg, Lt, n, nocc, d.n_core, f);
  k_scalars<<<1, 256, 0, st>>>((const double2*)in->h, G, n, d.n_core, epsh, EO);
  for (size_t li = 0; li < P->lists.size(); ++li) {
    DevList L = dev_list(P, (int)li, ws);
    if (L.n == 0) continue;
    k_unrank<<<blocks(L.n), 256, 0, st>>>(L, P->das, binom);
    k_eA<<<blocks(L.n), 256, 0, st>>>(L, epsh, G, n, sp.a0);
    k_U<<<blocks((int64_t)(P->nx + 1) * L.n), 256, 0, st>>>(L, sp, G);
  }
  // integral blocks
  const int modes[E2_NCLASS] = {-1, -1, INT_W02, -1, INT_W11, INT_W12, INT_W20, INT_W21, -1};
  const int cols[E2_NCLASS] = {0, 0, P->ntp, 0, 1 + na * na, na, P->ntp, na, 0};
  for (int c = 0; c < E2_NCLASS; ++c) {
    if (modes[c] < 0 || P->M[c] == 0) continue;
    k_rows<<<blocks(P->M[c]), 256, 0, st>>>(c, sp, epsh, G, P->M[c], (RowInfo*)W(P->o_rows[c]));
    k_integrals<<<blocks(P->M[c] * P->Kp[c]), 256, 0, st>>>(modes[c], sp, Bo, wt, Lt, f, P->M[c], cols[c], P->Kp[c],
                                                             W(P->o_W[c]));
  }
  if (P->part_cnt[8] > 0)
    k_integrals<<<blocks(P->ncp * P->nvp), 256, 0, st>>>(INT_G22, sp, Bo, wt, Lt, f, P->ncp, (int)P->nvp, (int)P->nvp,
                                                         W(P->o_G22));
  if (P->part_cnt[1] > 0)
    k_integrals<<<blocks((int64_t)P->nvc * na * P->ntp), 256, 0, st>>>(INT_X01, sp, Bo, wt, Lt, f, P->nvc, na * P->ntp,
                                                                       na * P->ntp, W(P->o_X01));
  if (P->part_cnt[3] > 0)
    k_integrals<<<blocks((int64_t)P->ncc * P->ntp * na), 256, 0, st>>>(INT_X10, sp, Bo, wt, Lt, f, P->ncc, P->ntp * na,
                                                                       P->ntp * na, W(P->o_X10));
  if (P->ntp > 0)
    k_integrals<<<blocks((int64_t)P->ntp * P->ntp), 256, 0, st>>>(INT_X00, sp, Bo, wt, Lt, f, P->ntp, P->ntp, P->ntp,
                                                                  W(P->o_X00));
  // per root: coupling tensors, E0, classes
  const DevList LP = dev_list(P, P->listP, ws);
  DevList Lc[E2_NCLASS];
  for (int c = 0; c < E2_NCLASS; ++c) Lc[c] = dev_list(P, P->list_of[c], ws);
  double* part = (double*)W(P->o_part);
  for (int r = 0; r < R; ++r) {
    const double2* c = (const double2*)in->c + (int64_t)r * LP.n;
    unsigned char* dr = ws + P->d_stride * r;
    double2* DT = (double2*)(dr + P->o_DT);
    double2* DTD = (double2*)(dr + P->o_DTD);
    double2* DTU = (double2*)(dr + P->o_DTU);
    double2* DTDUD = (double2*)(dr + P->o_DTDUD);
    double2* DTDU = (double2*)(dr + P->o_DTDU);
    struct T {
      int fam, cls, Kp;
      double2* out;
    } tabs[5] = {{FAM_T, 5, P->KpT, DT}, {FAM_TD, 7, P->KpT, DTD}, {FAM_TU, 2, P->KpTU, DTU},
                 {FAM_TDUD, 6, P->KpTU, DTDUD}, {FAM_TDU, 4, P->Kp11, DTDU}};
    for (const T& t : tabs) {
      const DevList& L = Lc[t.cls];
      if (L.n == 0) continue;
      k_dtable<<<blocks((int64_t)t.Kp * L.n), 256, 0, st>>>(t.fam, L, LP, P->das, binom, c, t.Kp, t.out);
    }
    double2* g1 = (double2*)(ws + P->o_g1 + P->g_stride * r);
    double2* g2 = (double2*)(ws + P->o_g2 + P->g_stride * r);
    k_gram<<<1 + na * na, 256, 0, st>>>(DTDU, DTDU, Lc[4].n, 1 + na * na, g1);
    if (P->ntp > 0 && Lc[2].n > 0) k_gram<<<P->ntp * P->ntp, 256, 0, st>>>(DTU, DTU, Lc[2].n, P->ntp, g2);
    else cudaMemsetAsync(g2, 0, 16 * (size_t)std::max(P->ntp * P->ntp, 1), st);
    k_e0<<<1, 256, 0, st>>>(g1, g2, f, (const double2*)W(P->o_X00), sp, P->ntp, EO, E0p + r, E0d + r);

    double* pr = part;
    auto poff = [&](int cls) { return pr + P->part_off[r * E2_NCLASS + cls]; };
    const double2* Dfor[E2_NCLASS] = {nullptr, nullptr, DTU, nullptr, DTDU, DT, DTDUD, DTD, nullptr};
    for (int cls : {2, 5, 7, 4, 6}) {
      if (P->part_cnt[cls] == 0) continue;
      const DevList& L = Lc[cls];
      dim3 grid((unsigned)((P->M[cls] + 63) / 64), (unsigned)((L.n + 63) / 64));
      k_class_gemm<<<grid, 256, 0, st>>>((const double2*)W(P->o_W[cls]), Dfor[cls], P->M[cls], L.n, P->Kp[cls],
                                         (const RowInfo*)W(P->o_rows[cls]), L.U, L.eA, E0p + r, b, poff(cls));
    }
    if (P->part_cnt[8] > 0) {
      const DevList& L = Lc[8];
      dim3 grid(blocks(L.n), (unsigned)(P->nvb * (P->nvb + 1) / 2), (unsigned)P->ncp);
      k_class22<<<grid, 256, 0, st>>>(L, sp, c, (const double*)W(P->o_G22), epsh, G, E0p + r, b, P->nvb, poff(8));
    }
    if (P->part_cnt[1] > 0) {
      dim3 grid(blocks(Lc[1].n), (unsigned)P->nvc);
      k_class01<<<grid, 256, 0, st>>>(Lc[1], Lc[5], Lc[2], P->das, sp, binom, DT, DTU, (const double2*)W(P->o_X01), f,
                                      epsh, E0p + r, b, poff(1));
    }
    if (P->part_cnt[3] > 0) {
      dim3 grid(blocks(Lc[3].n), (unsigned)P->ncc);
      k_class10<<<grid, 256, 0, st>>>(Lc[3], Lc[7], Lc[5], P->das, sp, binom, DTD, DT, (const double2*)W(P->o_X10), f,
                                      epsh, E0p + r, b, poff(3));
    }
    if (P->part_cnt[0] > 0)
      k_class00<<<blocks(Lc[0].n), 256, 0, st>>>(Lc[0], Lc[4], Lc[2], P->das, sp, binom, DTDU, DTU,
                                                 (const double2*)W(P->o_X00), f, E0p + r, b, poff(0));
  }
  double* e2c = E2_class ? E2_class : (double*)W(P->o_e2c);
  k_reduce<<<R * E2_NCLASS, 256, 0, st>>>(part, (const int64_t*)W(P->o_partoff), (const int64_t*)W(P->o_partcnt),
                                          (const double2*)(ws + P->o_g1), (int)(P->g_stride / 16), R, e2c);
  k_finalize<<<1, 32, 0, st>>>(e2c, R, E2, E0d, E0);
  if (cudaGetLastError() != cudaSuccess) return E2_ERR_CUDA;
  return E2_OK;
}

}  // extern "C"
