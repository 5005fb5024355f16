// C ABI: host plan (occupation patterns, string lists, workspace layout) and
// the stream-ordered launch sequence of e2_forward.  No device allocation.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <new>
#include <queue>
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

// Column tiles of a dense class with a compacted contraction (see ColTiles).
struct ColPlan {
  bool built = false;
  std::vector<int32_t> perm;   // [tiles * 64] list index, -1 = padding
  std::vector<int32_t> tdesc;  // [tiles][4] {koff, klen, ktrue, 0}
  std::vector<int32_t> klist;  // [krows]
  std::vector<int32_t> pos;    // [tiles][Kp] compacted row of table row x in tile j, -1 if absent
  int64_t tiles = 0, krows = 0;
  int maxklen = 0;             // longest compacted contraction of a tile
  int gran = 8;                // contraction granularity of the tiles (4: a k = 4 tail step)
  int64_t gd_ctas = 0;         // sum over tiles of ceil(klen / 64)
  double ratio = 1.0;          // krows / (tiles * Kp): share of the dense contraction
  size_t o_perm = 0, o_tdesc = 0, o_klist = 0, o_pos = 0, o_Dc = 0;  // o_Dc: per-root D region
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

struct e2_batch;

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
  size_t o_vaY, o_vaZ, o_vaX, va_cap;
  size_t o_xYc, o_xZaa, o_x12, o_x01;
  size_t o_DT, o_DTD, o_DTU, o_DTDUD, o_DTDU;  // per-root stride below
  size_t d_stride;                              // bytes of one root's D tables
  bool multi_slot = false;                      // set while a batch uses the job: one slot per root
  size_t o_g1, o_g2, g_stride;                  // gram outputs per root
  size_t o_part, o_partoff, o_partcnt, o_e2c;
  int64_t part_cnt[E2_NCLASS];
  std::vector<int64_t> part_off;                // [n_roots][E2_NCLASS]
  std::vector<unsigned char> plan_blob;         // host image of the plan region
  // launch shapes of the sparse / elementwise classes
  int nvb;
  // optional CUDA events around each class kernel of root 0 (bench hooks)
  cudaEvent_t prof[2 * E2_NCLASS];
  bool prof_on = false;
  int64_t launches = 0;  // kernels enqueued by the last e2_forward
  // reference solver region
  int sv_mmax;
  size_t o_sV, o_sS, o_sX, o_sR, o_sD, o_sT, o_sG, o_sY, solve_bytes;
  // adjoint region
  size_t o_dstart;                   // first D table of the root-0 slot
  int64_t chunk_rows[E2_NCLASS];     // dense-class rows per adjoint chunk
  size_t o_gD, o_bT, o_bHrow, o_bHcol, o_bScalT, o_bHsum, o_bHA, o_bRowdot;
  size_t o_bGT, o_bGH, o_bGV, o_bC22p, o_bH22p, o_bV22, o_bC22, o_bGc, o_bSig, o_bGf, o_bNx, o_bNt, o_bNd, o_bScal;
  // factor gradient
  int64_t npair;
  size_t o_bGW[E2_NCLASS], o_bHm, o_bHocc, o_bZ, o_bZs, o_bGe, o_bGea, o_bNtt, o_bGG, o_bGt, o_bGh, o_bTsh;
  size_t o_bGX01, o_bGX10, o_bGX00, o_bR22, o_bHs22, o_bP22, o_bG22c, o_bGg22, o_bCs, o_bGB, o_bFtr, o_bGw, o_bRg;
  size_t o_bPart, bpart_bytes;  // split-K segments
  size_t tsh_bytes;
  size_t o_bGDc, o_bGWc, gwc_bytes;
  size_t bwd_bytes;
  // compacted column tiles of the dense classes and whether each class uses them
  ColPlan cplan[E2_NCLASS];
  bool use_cols[E2_NCLASS] = {};
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

// Active-local bitset of the k-subset of colex rank r (r = sum_j C(t_j, j)).
uint64_t colex_unrank_h(int64_t r, int k) {
  uint64_t bits = 0;
  for (int j = k; j >= 1; --j) {
    int t = j - 1;
    while (binom_h(t + 1, j) <= r) ++t;
    r -= binom_h(t, j);
    bits |= 1ull << t;
  }
  return bits;
}

// The strings of a list in address order (pattern blocks, subspace 1 fastest,
// colex inside each subspace): the order the device unranks them in.
std::vector<uint64_t> host_strings(const e2_problem* P, const HostList& L) {
  std::vector<uint64_t> out;
  out.reserve((size_t)L.n);
  for (const Pat& pt : L.pats) {
    const int64_t cnt = pattern_size(P, pt);
    for (int64_t g = 0; g < cnt; ++g) {
      int64_t r = g;
      uint64_t A = 0;
      for (int s = 0; s < P->d.n_das; ++s) {
        const int64_t cs = binom_h(P->das_size[s], pt[s]);
        A |= colex_unrank_h(r % cs, pt[s]) << P->das.off[s];
        r /= cs;
      }
      out.push_back(A);
    }
  }
  return out;
}

// Structural non-zero of coupling-table row x at string A (a necessary
// condition: the table entry is exactly zero when it fails).
bool table_nonzero(int fam, int na, uint64_t A, int x) {
  auto in = [&](int t) { return (A >> t) & 1ull; };
  switch (fam) {
    case FAM_T: return !in(x);
    case FAM_TD: return in(x);
    case FAM_TU:
    case FAM_TDUD: {
      int u = 1;
      while ((u + 1) * u / 2 <= x) ++u;
      const int t = x - u * (u - 1) / 2;
      return fam == FAM_TU ? (!in(t) && !in(u)) : (in(t) && in(u));
    }
    default: {  // FAM_TDU: row 0 is c_A, row 1 + t*na + u is a+_t a_u
      if (x == 0) return true;
      const int t = (x - 1) / na, u = (x - 1) % na;
      return t == u ? in(t) : (in(t) && !in(u));
    }
  }
}

// Column tiles of one dense class: strings grouped greedily by a shared
// 3-spinor set (occupied spinors for tables that need empty ones, empty
// spinors for those that need occupied ones), 64 to a tile, each tile keeping
// the table rows that are non-zero for some of its strings.
void build_colplan(e2_problem* P, int cls, int fam, int kvalid, int fs = 3, int gran = 8) {
  ColPlan& cp = P->cplan[cls];
  cp = ColPlan{};
  cp.gran = gran;
  const int li = P->list_of[cls];
  if (li < 0 || P->M[cls] == 0) return;
  const HostList& L = P->lists[li];
  const int na = P->na, Kp = P->Kp[cls];
  const std::vector<uint64_t> S = host_strings(P, L);
  const int64_t nS = (int64_t)S.size();
  const uint64_t full = na >= 64 ? ~0ull : ((1ull << na) - 1);
  const bool by_occ = (fam == FAM_T || fam == FAM_TU || fam == FAM_TDU);
  const int nkey = by_occ ? L.count : na - L.count;
  std::vector<int32_t> order;
  order.reserve((size_t)nS);
  if (nkey < fs || na < fs) {
    for (int64_t s = 0; s < nS; ++s) order.push_back((int32_t)s);
  } else {
    const int nsub = (int)binom_h(nkey, fs);
    const int64_t nF = binom_h(na, fs);
    std::vector<int32_t> fid((size_t)nS * nsub);
    std::vector<int64_t> fcnt((size_t)nF, 0);
    for (int64_t s = 0; s < nS; ++s) {
      const uint64_t key = by_occ ? S[s] : (~S[s] & full);
      int bits[64], nb = 0;
      for (uint64_t x = key; x; x &= x - 1) bits[nb++] = __builtin_ctzll(x);
      // every fs-subset of the key spinors, by colex rank
      int q = 0, idx[8];
      for (int i = 0; i < fs; ++i) idx[i] = i;
      for (;;) {
        int64_t f = 0;
        for (int i = 0; i < fs; ++i) f += binom_h(bits[idx[i]], i + 1);
        fid[(size_t)s * nsub + q++] = (int32_t)f;
        ++fcnt[f];
        int i = fs - 1;
        while (i >= 0 && idx[i] == nb - fs + i) --i;
        if (i < 0) break;
        ++idx[i];
        for (int j = i + 1; j < fs; ++j) idx[j] = idx[j - 1] + 1;
      }
    }
    std::vector<int64_t> boff((size_t)nF + 1, 0);
    for (int64_t f = 0; f < nF; ++f) boff[f + 1] = boff[f] + fcnt[f];
    std::vector<int32_t> bucket((size_t)boff[nF]);
    std::vector<int64_t> fill(boff.begin(), boff.end() - 1);
    for (int64_t s = 0; s < nS; ++s)
      for (int q = 0; q < nsub; ++q) bucket[fill[fid[(size_t)s * nsub + q]]++] = (int32_t)s;
    std::vector<int64_t> ptr(boff.begin(), boff.end() - 1);
    std::vector<char> alive((size_t)nS, 1);
    std::priority_queue<std::pair<int64_t, int64_t>> heap;  // (count, -F): largest, then smallest F
    for (int64_t f = 0; f < nF; ++f)
      if (fcnt[f] > 0) heap.push({fcnt[f], -f});
    int64_t left = nS;
    std::vector<int32_t> cur;
    while (left > 0 && !heap.empty()) {
      const auto top = heap.top();
      heap.pop();
      const int64_t f = -top.second;
      if (top.first != fcnt[f]) {
        if (fcnt[f] > 0) heap.push({fcnt[f], -f});
        continue;
      }
      while (ptr[f] < boff[f + 1] && (int)cur.size() < 64) {
        const int32_t s = bucket[ptr[f]++];
        if (!alive[s]) continue;
        alive[s] = 0;
        cur.push_back(s);
        --left;
        for (int q = 0; q < nsub; ++q) --fcnt[fid[(size_t)s * nsub + q]];
      }
      if ((int)cur.size() == 64 || left == 0) {
        std::sort(cur.begin(), cur.end());
        order.insert(order.end(), cur.begin(), cur.end());
        cur.clear();
      }
      if (fcnt[f] > 0) heap.push({fcnt[f], -f});
    }
    if (!cur.empty()) {
      std::sort(cur.begin(), cur.end());
      order.insert(order.end(), cur.begin(), cur.end());
    }
  }
  cp.tiles = (nS + 63) / 64;
  cp.perm.assign((size_t)cp.tiles * 64, -1);
  std::copy(order.begin(), order.end(), cp.perm.begin());
  const int words = (kvalid + 63) / 64;
  std::vector<uint64_t> mask((size_t)words);
  for (int64_t j = 0; j < cp.tiles; ++j) {
    std::fill(mask.begin(), mask.end(), 0ull);
    for (int c = 0; c < 64; ++c) {
      const int32_t s = cp.perm[j * 64 + c];
      if (s < 0) continue;
      for (int x = 0; x < kvalid; ++x)
        if (!((mask[x >> 6] >> (x & 63)) & 1ull) && table_nonzero(fam, na, S[s], x)) mask[x >> 6] |= 1ull << (x & 63);
    }
    const int koff = (int)cp.klist.size();
    int ktrue = 0;
    for (int x = 0; x < kvalid; ++x)
      if ((mask[x >> 6] >> (x & 63)) & 1ull) {
        cp.klist.push_back(x);
        ++ktrue;
      }
    const int klen = std::max(gran, (ktrue + gran - 1) / gran * gran);
    for (int x = ktrue; x < klen; ++x) cp.klist.push_back(0);
    cp.tdesc.insert(cp.tdesc.end(), {koff, klen, ktrue, 0});
    cp.maxklen = std::max(cp.maxklen, klen);
    cp.gd_ctas += (klen + 79) / 80;  // 64 x 80 product tiles of the compacted backward products
  }
  cp.pos.assign((size_t)cp.tiles * Kp, -1);
  for (int64_t j = 0; j < cp.tiles; ++j)
    for (int k = 0; k < cp.tdesc[4 * j + 2]; ++k) cp.pos[(size_t)j * Kp + cp.klist[cp.tdesc[4 * j] + k]] = k;
  cp.krows = (int64_t)cp.klist.size();
  cp.ratio = (double)cp.krows / ((double)cp.tiles * Kp);
  cp.built = true;
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
  // compacted column tiles where the coupling tables are mostly structural
  // zeros: D^{tu} (class (0,2)), D^{t+u+} (class (2,0)), D^{t+u} (class (1,1))
  build_colplan(P, 2, FAM_TU, P->ntp);
  build_colplan(P, 6, FAM_TDUD, P->ntp);
  build_colplan(P, 4, FAM_TDU, 1 + P->na * P->na);
  // D^t (class (1,2)): strings sharing four occupied spinors leave at most
  // n_act - 4 non-zero rows; a k = 4 tail step turns that into work saved
  build_colplan(P, 5, FAM_T, P->na, 4, 4);
  for (int c = 0; c < E2_NCLASS; ++c) P->use_cols[c] = P->cplan[c].built && P->cplan[c].ratio < 0.85;

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
  for (ColPlan& cp : P->cplan) {
    if (!cp.built) continue;
    cp.o_perm = ws.take(sizeof(int32_t) * cp.perm.size());
    cp.o_tdesc = ws.take(sizeof(int32_t) * cp.tdesc.size());
    cp.o_klist = ws.take(sizeof(int32_t) * cp.klist.size());
    cp.o_pos = ws.take(sizeof(int32_t) * cp.pos.size());
  }
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
  P->o_dstart = dstart;
  P->o_DT = ws.take(16 * (size_t)P->KpT * std::max<int64_t>(lsize(5), 1));
  P->o_DTD = ws.take(16 * (size_t)P->KpT * std::max<int64_t>(lsize(7), 1));
  P->o_DTU = ws.take(16 * (size_t)P->KpTU * std::max<int64_t>(lsize(2), 1));
  P->o_DTDUD = ws.take(16 * (size_t)P->KpTU * std::max<int64_t>(lsize(6), 1));
  P->o_DTDU = ws.take(16 * (size_t)P->Kp11 * std::max<int64_t>(lsize(4), 1));
  for (ColPlan& cp : P->cplan)
    if (cp.built) cp.o_Dc = ws.take(16 * (size_t)cp.krows * 64);
  P->d_stride = ws.top - dstart;
  // one slot: the forward and backward build and consume each root's tables
  // in turn on one stream; a batch, which holds every root's tables until its
  // single launch, appends R - 1 more slots to each job's region
  ws.top = dstart + P->d_stride;
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
  // Scratch of the integrals formed as products over the factor index:
  // weighted and plain (virtual, active) factor columns, (virtual, core) and
  // active-pair columns, (ai|bt), (av|uw) and a stripe of (at|bu).  It lies
  // over the D tables and partials, which are written only after the
  // integrals are formed; the stripe holds the whole lower triangle when that
  // takes at most 1 GiB (else what is left there, at least 8 virtuals of
  // rows), extending the workspace as needed.
  {
    const int64_t nva = (int64_t)P->nvc * P->na;
    const size_t yb = 16 * (size_t)std::max<int64_t>(nva * Lt, 1);
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    P->o_vaY = P->o_dstart;
    P->o_vaZ = P->o_vaY + al(yb);
    // (virtual, core) and active-pair factor columns, (ai|bt) and (av|uw)
    P->o_xYc = P->o_vaZ + al(yb);
    P->o_xZaa = P->o_xYc + al(16 * (size_t)std::max<int64_t>((int64_t)P->nvc * P->ncc * Lt, 1));
    P->o_x12 = P->o_xZaa + al(16 * (size_t)std::max<int64_t>((int64_t)P->na * P->na * Lt, 1));
    P->o_x01 = P->o_x12 + al(16 * (size_t)std::max<int64_t>((int64_t)P->nvc * P->ncc * nva, 1));
    P->o_vaX = P->o_x01 + al(16 * (size_t)std::max<int64_t>(nva * P->na * P->na, 1));
    const size_t full = 16 * (size_t)std::max<int64_t>(nva * nva, 1);
    const size_t least = 16 * (size_t)std::max<int64_t>((int64_t)std::min(8, P->nvc) * P->na * nva, 1);
    const size_t room = ws.top > P->o_vaX ? ws.top - P->o_vaX : 0;
    // the whole lower triangle in one product when it takes at most 1 GiB
    P->va_cap = std::min(full, std::max(std::max(least, room), std::min(full, size_t(1) << 30)));
    ws.top = std::max(ws.top, P->o_vaX + P->va_cap);
  }
  P->ws_bytes = ws.top;
  // reference solver (block Davidson) on top of the forward layout
  const int64_t np_ = P->lists[P->listP].n;
  P->sv_mmax = (int)std::min<int64_t>(np_, 10 * R + 10);
  P->o_sV = ws.take(16 * (size_t)P->sv_mmax * np_);
  P->o_sS = ws.take(16 * (size_t)P->sv_mmax * np_);
  P->o_sX = ws.take(16 * (size_t)R * np_);
  P->o_sR = ws.take(16 * (size_t)R * np_);
  P->o_sD = ws.take(16 * (size_t)R * np_);
  P->o_sT = ws.take(16 * (size_t)R * np_);
  P->o_sG = ws.take(16 * (size_t)P->sv_mmax * P->sv_mmax);
  P->o_sY = ws.take(16 * (size_t)P->sv_mmax * std::max(R, 1));
  P->solve_bytes = ws.top;
  // adjoint region on top of the solver layout (the forward one is its prefix)
  {
    const size_t tbudget = size_t(4) << 30, gwbudget = size_t(8) << 30;
    size_t tmax = 16, hrow = 8, hcol = 8, scalt = 16, hsum = 8, hA = 8, gdc = 16, gwc = 16;
    for (int c : {2, 5, 7, 4, 6}) {
      const int64_t Mc = P->M[c], Nc = lsize(c);
      P->chunk_rows[c] = 0;
      if (Mc == 0 || Nc == 0) continue;
      int64_t rows_fit = (int64_t)(tbudget / (16 * (size_t)Nc)) / 64 * 64;
      if (P->cplan[c].built)  // compacted Gamma_W of a chunk: rows x compacted columns
        rows_fit = std::min<int64_t>(rows_fit, (int64_t)(gwbudget / (16 * (size_t)P->cplan[c].krows)) / 64 * 64);
      rows_fit = std::max<int64_t>(64, rows_fit);
      P->chunk_rows[c] = std::min<int64_t>(rows_fit, (Mc + 63) / 64 * 64);
      const int64_t rt = (Mc + 63) / 64, ct = (Nc + 63) / 64;
      tmax = std::max(tmax, (size_t)16 * P->chunk_rows[c] * Nc);
      if (P->cplan[c].built) {
        gdc = std::max(gdc, (size_t)16 * P->cplan[c].krows * 64);
        gwc = std::max(gwc, (size_t)16 * P->chunk_rows[c] * P->cplan[c].krows);
      }
      hrow = std::max(hrow, (size_t)8 * Mc * ct);
      hcol = std::max(hcol, (size_t)8 * rt * Nc);
      scalt = std::max(scalt, (size_t)16 * rt * ct);
      hsum = std::max(hsum, (size_t)8 * Mc);
    }
    for (size_t li = 0; li < P->lists.size(); ++li) hA = std::max(hA, (size_t)8 * P->lists[li].n);
    size_t gmax = 8;
    for (int c : {1, 3, 0})
      if (P->list_of[c] >= 0) gmax = std::max(gmax, (size_t)P->M[c] * P->lists[P->list_of[c]].n);
    const int64_t nyb = (int64_t)P->nvb * (P->nvb + 1) / 2;
    const int64_t np22 = lsize(8), xb22 = (np22 + 255) / 256;
    const size_t yz = (size_t)std::max<int64_t>(1, nyb * P->ncp);
    P->o_gD = ws.take(P->d_stride);
    P->o_bT = ws.take(tmax);
    P->o_bGDc = ws.take(gdc);  // compacted Gamma_D / Gamma_W of a column-tiled class
    P->o_bGWc = ws.take(gwc);
    P->gwc_bytes = gwc;
    P->o_bHrow = ws.take(hrow);
    P->o_bHcol = ws.take(hcol);
    P->o_bScalT = ws.take(scalt);
    P->o_bHsum = ws.take(hsum);
    P->o_bHA = ws.take(hA);
    P->o_bRowdot = ws.take(16 * (size_t)std::max<int64_t>(P->M[4], 1));
    P->o_bGT = ws.take(16 * gmax);
    P->o_bGH = ws.take(8 * gmax);
    P->o_bGV = ws.take(8 * gmax);
    P->o_bC22p = ws.take(8 * yz * std::max<int64_t>(np22, 1));
    P->o_bH22p = ws.take(8 * yz * std::max<int64_t>(np22, 1));
    P->o_bV22 = ws.take(8 * 19 * yz * std::max<int64_t>(xb22, 1));
    P->o_bC22 = ws.take(8 * (size_t)std::max<int64_t>(np_, 1));
    P->o_bGc = ws.take(16 * (size_t)np_);
    P->o_bSig = ws.take(16 * (size_t)np_);
    P->o_bGf = ws.take(16 * (size_t)P->n * P->nocc);
    P->o_bNx = ws.take(8 * (size_t)(P->nx + 1));
    P->o_bNt = ws.take(8 * (size_t)std::max(P->na, 1));
    P->o_bNd = ws.take(8 * (size_t)P->n);
    P->o_bScal = ws.take(16);
    // factor gradient
    const int64_t npair = (int64_t)P->n * P->nocc;
    P->npair = npair;
    size_t hm = 8, hocc = 8, zz = 8, tsh = 16;
    for (int c = 0; c < E2_NCLASS; ++c) P->o_bGW[c] = 0;
    for (int c : {2, 5, 7, 4, 6}) {
      const int64_t Mc = P->M[c], Nc = lsize(c);
      if (Mc == 0 || Nc == 0) continue;
      P->o_bGW[c] = ws.take(16 * (size_t)Mc * P->Kp[c]);
      hm = std::max(hm, (size_t)8 * P->chunk_rows[c] * Nc);
      hocc = std::max(hocc, (size_t)8 * Mc * P->na);
      zz = std::max(zz, (size_t)8 * Mc * P->nx);
    }
    const int64_t M22 = P->ncp * P->nvp;
    hocc = std::max(hocc, (size_t)8 * std::max<int64_t>(M22, 1) * P->na);
    zz = std::max(zz, (size_t)8 * std::max<int64_t>(M22, 1) * P->nx);
    for (int c : {1, 3, 0})
      if (P->list_of[c] >= 0) {
        hocc = std::max(hocc, (size_t)8 * P->M[c] * P->na);
        zz = std::max(zz, (size_t)8 * P->M[c] * P->nx);
      }
    {  // shifted amplitudes of the gather classes: all shifts of a row chunk
      const size_t n01 = 16 * (size_t)P->na * std::max<int64_t>(lsize(2), 1);
      const size_t n10 = 16 * (size_t)std::max(P->ntp, 1) * std::max<int64_t>(lsize(5), 1);
      const size_t n00 = 16 * (size_t)std::max(P->ntp, 1) * std::max<int64_t>(lsize(2), 1);
      const size_t one = std::max(n01, std::max(n10, n00));
      const size_t all = std::max(n01 * std::max(P->nvc, 1), std::max(n10 * std::max(P->ncc, 1), n00));
      tsh = std::max(one, std::min(all, size_t(1) << 30));
      P->tsh_bytes = tsh;
    }
    P->o_bHm = ws.take(hm);
    P->o_bHocc = ws.take(hocc);
    P->o_bZ = ws.take(zz);
    P->o_bZs = ws.take(zz);
    P->o_bRg = ws.take(sizeof(RowInfo) * (size_t)std::max<int64_t>(std::max(P->nvc, P->ncc), 1));
    P->o_bGe = ws.take(8 * (size_t)std::max(P->nx, 1) * std::max(P->nx, 1));
    P->o_bGea = ws.take(8 * (size_t)std::max(P->nx, 1) * std::max(P->na, 1));
    P->o_bNtt = ws.take(8 * (size_t)P->na * P->na);
    P->o_bGG = ws.take(8 * (size_t)P->n * P->n);
    P->o_bGt = ws.take(16 * (size_t)npair * npair);
    P->o_bGh = ws.take(16 * (size_t)npair * npair);
    P->o_bTsh = ws.take(tsh);
    P->o_bGX01 = ws.take(16 * (size_t)std::max<int64_t>((int64_t)P->nvc * P->na * P->ntp, 1));
    P->o_bGX10 = ws.take(16 * (size_t)std::max<int64_t>((int64_t)P->ncc * P->ntp * P->na, 1));
    P->o_bGX00 = ws.take(16 * (size_t)std::max<int64_t>((int64_t)P->ntp * P->ntp, 1));
    P->o_bR22 = ws.take(sizeof(RowInfo) * (size_t)std::max<int64_t>(M22, 1));
    P->o_bHs22 = ws.take(8 * (size_t)std::max<int64_t>(M22, 1));
    P->o_bP22 = ws.take(8 * (size_t)std::max<int64_t>(M22, 1));
    P->o_bG22c = ws.take(16 * (size_t)std::max<int64_t>(M22, 1));
    P->o_bGg22 = ws.take(16 * (size_t)std::max<int64_t>(M22, 1));
    P->o_bCs = ws.take(16 * (size_t)Lt * npair);
    P->o_bGB = ws.take(16 * (size_t)Lt * P->n * P->n);
    P->o_bFtr = ws.take(16 * (size_t)std::max(Lt, 1));
    P->o_bGw = ws.take(8 * (size_t)std::max(Lt, 1));
    P->bpart_bytes = size_t(512) << 20;
    P->o_bPart = ws.take(P->bpart_bytes);
    P->bwd_bytes = ws.top;
  }

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
  for (const ColPlan& cp : P->cplan) {
    if (!cp.built) continue;
    put(P->plan_blob, rel(cp.o_perm), cp.perm.data(), cp.perm.size());
    put(P->plan_blob, rel(cp.o_tdesc), cp.tdesc.data(), cp.tdesc.size());
    put(P->plan_blob, rel(cp.o_klist), cp.klist.data(), cp.klist.size());
    put(P->plan_blob, rel(cp.o_pos), cp.pos.data(), cp.pos.size());
  }
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

// kernels enqueued by the current host thread (read back as the count of one call)
thread_local int64_t g_launches = 0;

using cd = std::complex<double>;

// Cyclic Jacobi for a complex Hermitian matrix A (n x n, row-major):
// eigenvalues ascending in w, eigenvectors in the columns of V (row-major).
// Each rotation U = [[c, s e^{i phi}], [-s e^{-i phi}, c]] in the (p,q) plane
// zeroes A_pq = g e^{i phi}: t = s/c solves t^2 + 2 tau t - 1 = 0,
// tau = (A_qq - A_pp) / (2 g), smaller root.
void herm_eig(int n, std::vector<cd> A, std::vector<double>& w, std::vector<cd>& V) {
  V.assign((size_t)n * n, cd(0.0, 0.0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int p = 0; p < n; ++p) {
      dia += std::norm(A[(size_t)p * n + p]);
      for (int q = p + 1; q < n; ++q) off += std::norm(A[(size_t)p * n + q]);
    }
    if (off <= 1e-32 * (dia + 1e-300)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const cd apq = A[(size_t)p * n + q];
        const double g = std::abs(apq);
        if (g < 1e-300) continue;
        const cd ph = apq / g;
        const double a = A[(size_t)p * n + p].real(), bq = A[(size_t)q * n + q].real();
        const double tau = (bq - a) / (2.0 * g);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
        const cd u00 = cs, u01 = sn * ph, u10 = -sn * std::conj(ph), u11 = cs;
        for (int r = 0; r < n; ++r) {  // A <- A U, V <- V U
          cd x = A[(size_t)r * n + p], y = A[(size_t)r * n + q];
          A[(size_t)r * n + p] = x * u00 + y * u10;
          A[(size_t)r * n + q] = x * u01 + y * u11;
          x = V[(size_t)r * n + p];
          y = V[(size_t)r * n + q];
          V[(size_t)r * n + p] = x * u00 + y * u10;
          V[(size_t)r * n + q] = x * u01 + y * u11;
        }
        for (int r = 0; r < n; ++r) {  // A <- U^H A
          cd x = A[(size_t)p * n + r], y = A[(size_t)q * n + r];
          A[(size_t)p * n + r] = std::conj(u00) * x + std::conj(u10) * y;
          A[(size_t)q * n + r] = std::conj(u01) * x + std::conj(u11) * y;
        }
      }
  }
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return A[(size_t)x * n + x].real() < A[(size_t)y * n + y].real(); });
  w.resize(n);
  std::vector<cd> Vs((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = A[(size_t)ord[j] * n + ord[j]].real();
    for (int i = 0; i < n; ++i) Vs[(size_t)i * n + j] = V[(size_t)i * n + ord[j]];
  }
  V.swap(Vs);
}

struct Ctx {
  const int64_t* binom;
  double *G, *epsh, *EO, *E0p, *E0d, *dg, *wt;
  double2 *Bo, *f;
  DevSpace sp;
};

Ctx ctx(const e2_problem* P, unsigned char* ws) {
  Ctx X;
  X.binom = (const int64_t*)(ws + P->o_binom);
  X.G = (double*)(ws + P->o_G);
  X.epsh = (double*)(ws + P->o_epsh);
  X.EO = (double*)(ws + P->o_EO);
  X.E0p = (double*)(ws + P->o_E0p);
  X.E0d = (double*)(ws + P->o_E0);
  X.dg = (double*)(ws + P->o_dg);
  X.wt = (double*)(ws + P->o_wt);
  X.Bo = (double2*)(ws + P->o_Bo);
  X.f = (double2*)(ws + P->o_f);
  DevSpace& sp = X.sp;
  sp.n = P->n;
  sp.n_core = P->d.n_core;
  sp.n_act = P->na;
  sp.n_virt = P->d.n_virt;
  sp.n_occ = P->nocc;
  sp.a0 = P->d.n_core;
  sp.v0 = P->nocc;
  sp.ncc = P->ncc;
  sp.nvc = P->nvc;
  sp.nx = P->nx;
  sp.cc = (const int32_t*)(ws + P->o_cc);
  sp.vc = (const int32_t*)(ws + P->o_vc);
  return X;
}

struct Tabs {
  double2 *DT, *DTD, *DTU, *DTDUD, *DTDU;
};

// Base of root r's D-table slot (offsets o_DT... apply to it): slot 0 inside
// the layout, or for a batch slot r >= 1 after the job's forward layout.
unsigned char* slot_base(const e2_problem* P, unsigned char* ws, int r) {
  if (!P->multi_slot || r == 0) return ws;
  return ws + P->ws_bytes + (size_t)(r - 1) * P->d_stride - P->o_dstart;
}

Tabs tables(const e2_problem* P, unsigned char* ws, int r) {
  unsigned char* dr = slot_base(P, ws, r);
  return Tabs{(double2*)(dr + P->o_DT), (double2*)(dr + P->o_DTD), (double2*)(dr + P->o_DTU),
              (double2*)(dr + P->o_DTDUD), (double2*)(dr + P->o_DTDU)};
}

// Column tiles of class cls for root r (plain columns unless the class uses them).
ColTiles col_tiles(const e2_problem* P, unsigned char* ws, int r, int cls) {
  if (!P->use_cols[cls]) return ColTiles{nullptr, nullptr, nullptr, nullptr};
  const ColPlan& cp = P->cplan[cls];
  return ColTiles{(const int32_t*)(ws + cp.o_perm), (const int4*)(ws + cp.o_tdesc), (const int32_t*)(ws + cp.o_klist),
                  (const double2*)(slot_base(P, ws, r) + cp.o_Dc)};
}

// Coupling tensors D^x_A = <A|x|c> of one reference vector c; `all` = false
// builds only the two that the active sigma needs.
void build_tables(const e2_problem* P, unsigned char* ws, cudaStream_t st, const double2* c, const Tabs& T, bool all) {
  const DevList LP = dev_list(P, P->listP, ws);
  const Ctx X = ctx(P, ws);
  struct Spec {
    int fam, cls, Kp;
    double2* out;
  } tabs[5] = {{FAM_TU, 2, P->KpTU, T.DTU}, {FAM_TDU, 4, P->Kp11, T.DTDU}, {FAM_T, 5, P->KpT, T.DT},
               {FAM_TD, 7, P->KpT, T.DTD}, {FAM_TDUD, 6, P->KpTU, T.DTDUD}};
  for (int k = 0; k < (all ? 5 : 2); ++k) {
    const Spec& t = tabs[k];
    const DevList L = dev_list(P, P->list_of[t.cls], ws);
    if (L.n == 0) continue;
    (k_dtable<<<blocks((int64_t)t.Kp * L.n), 256, 0, st>>>(t.fam, L, LP, P->das, X.binom, c, t.Kp, t.out), ++g_launches);
  }
}

// Scratch for split-K segments of the GEMM helpers (set while a pass that
// owns such a region runs; null: no split).
thread_local void* g_splitk = nullptr;
thread_local size_t g_splitk_bytes = 0;

// Segments for a product with `tiles` output tiles (one CTA per SM, 148 SMs)
// and contraction K: the count (at most 64, at least 256 of K each) that
// minimises waves / segments, i.e. the time of a wave-quantised launch whose
// CTAs each take K / segments; ties go to fewer segments.
int splitk_segments(int64_t tiles, int64_t K, size_t seg_bytes) {
  if (!g_splitk || K < 512) return 1;
  const int64_t slots = 148;
  int64_t nmax = std::min<int64_t>(64, K / 256);
  nmax = std::min<int64_t>(nmax, (int64_t)(g_splitk_bytes / std::max<size_t>(seg_bytes, 1)));
  int best = 1;
  double tbest = (double)((tiles + slots - 1) / slots);
  for (int64_t n = 2; n <= nmax; ++n) {
    const double t = (double)((tiles * n + slots - 1) / slots) / (double)n;
    if (t < 0.97 * tbest) {
      tbest = t;
      best = (int)n;
    }
  }
  return best;
}

// C(m,n) = beta C(m,n) + sum_k opA(m,k) opB(k,n) (real, tensor pipe), C row-major
// with leading dimension ldc = N when split.
void dgemm(cudaStream_t st, int64_t M, int64_t N, int64_t K, const double* A, int64_t sam, int64_t sak,
           const double* B, int64_t sbk, int64_t sbn, double* C, int64_t ldc, int beta) {
  if (M <= 0 || N <= 0) return;
  const int64_t tiles = ((M + 63) / 64) * ((N + 63) / 64);
  const int nseg = ldc == N ? splitk_segments(tiles, K, 8 * (size_t)M * N) : 1;  // segments dense in C's layout
  const int64_t kseg = (K + nseg - 1) / nseg;
  dim3 grid((unsigned)((M + 63) / 64), (unsigned)((N + 63) / 64), (unsigned)nseg);
  if (nseg == 1) {
    (k_dgemm<<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, beta, kseg, 0), ++g_launches);
    return;
  }
  double* part = (double*)g_splitk;
  (k_dgemm<<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, part, ldc, 0, kseg, M * N), ++g_launches);
  if (!beta) cudaMemsetAsync(C, 0, 8 * (size_t)M * N, st);
  (k_dacc<<<blocks(M * N), 256, 0, st>>>(part, nseg, M * N, M * N, C), ++g_launches);
}

// C(m,n) = beta C(m,n) + sum_k opA(m,k) opB(k,n) (complex, tensor pipe), C(m,n)
// at C[m*csm + n*csn].  Tile width bn = 64 or 16.  With `part` given and few
// output tiles, K is split into segments summed in a fixed order (the output
// region C[0 .. M*N) must then be dense in C's layout).
void zgemm(cudaStream_t st, int64_t M, int64_t N, int64_t K, const double2* A, int64_t sam, int64_t sak, int conjA,
           const double2* B, int64_t sbk, int64_t sbn, int conjB, double2* C, int64_t csm, int64_t csn, int beta,
           int bn = 64) {
  if (M <= 0 || N <= 0) return;
  const int bm = bn == 16 ? 128 : 64;  // tiles 64 x 64 or 128 x 16
  const int64_t tiles = ((M + bm - 1) / bm) * ((N + bn - 1) / bn);
  const int nseg = splitk_segments(tiles, K, 16 * (size_t)M * N);
  const int64_t kseg = (K + nseg - 1) / nseg;
  dim3 grid((unsigned)((M + bm - 1) / bm), (unsigned)((N + bn - 1) / bn), (unsigned)nseg);
  // split: segment z is written dense row-major at scratch + z*M*N, then summed into C
  double2* out = nseg > 1 ? (double2*)g_splitk : C;
  const int64_t om = nseg > 1 ? N : csm, on = nseg > 1 ? 1 : csn;
  const int b = nseg > 1 ? 0 : beta;
  const int64_t czs = M * N;
  if (bn == 16)
    (k_zgemm16<<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, conjA, B, sbk, sbn, conjB, out, om, on, b, kseg, czs, -1),
     ++g_launches);
  else
    (k_zgemm64<<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, conjA, B, sbk, sbn, conjB, out, om, on, b, kseg, czs, -1),
     ++g_launches);
  if (nseg > 1) (k_zacc<<<blocks(M * N), 256, 0, st>>>(out, nseg, czs, M, N, C, csm, csn, beta), ++g_launches);
}

// Everything that depends only on the Hamiltonian and the partition:
// binomials, compact factors, G, eps^, f, E_O, string lists with e_A and U,
// and the active two-electron block <tu||vw>.
e2_status setup_common(e2_problem* P, const e2_inputs* in, unsigned char* ws, cudaStream_t st, bool upload = true) {
  const e2_desc& d = P->d;
  const int n = P->n, nocc = P->nocc, Lt = d.L_coulomb + d.L_extra;
  Ctx X = ctx(P, ws);
  if (upload &&
      cudaMemcpyAsync(ws + P->o_plan, P->plan_blob.data(), P->plan_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return E2_ERR_CUDA;
  (k_binom<<<1, 256, 0, st>>>((int64_t*)(ws + P->o_binom)), ++g_launches);
  {
    int64_t tot = (int64_t)Lt * n * nocc;
    unsigned g = (unsigned)std::min<int64_t>(blocks(tot), 148 * 64);
    (k_extract<<<g, 256, 0, st>>>((const double2*)in->B_c, (const double2*)in->B_x, in->w_x, in->lambda, d.L_coulomb,
                                 d.L_extra, n, nocc, X.Bo, X.wt, X.dg), ++g_launches);
  }
  (k_G<<<blocks((int64_t)n * n), 256, 0, st>>>((const double2*)in->B_c, (const double2*)in->B_x, X.wt, X.dg, d.L_coulomb,
                                              d.L_extra, n, X.G), ++g_launches);
  (k_fock<<<blocks((int64_t)n * nocc), 256, 0, st>>>((const double2*)in->h, X.Bo, X.wt, X.dg, Lt, n, nocc, d.n_core, X.f), ++g_launches);
  (k_scalars<<<1, 256, 0, st>>>((const double2*)in->h, X.G, n, d.n_core, X.epsh, X.EO), ++g_launches);
  for (size_t li = 0; li < P->lists.size(); ++li) {
    DevList L = dev_list(P, (int)li, ws);
    if (L.n == 0) continue;
    (k_unrank<<<blocks(L.n), 256, 0, st>>>(L, P->das, X.binom), ++g_launches);
    (k_eA<<<blocks(L.n), 256, 0, st>>>(L, X.epsh, X.G, n, X.sp.a0), ++g_launches);
    (k_U<<<blocks((int64_t)(P->nx + 1) * L.n), 256, 0, st>>>(L, X.sp, X.G), ++g_launches);
  }
  if (P->ntp > 0)
    (k_integrals<<<blocks((int64_t)P->ntp * P->ntp), 256, 0, st>>>(INT_X00, X.sp, X.Bo, X.wt, Lt, X.f, P->ntp, P->ntp,
                                                                  P->ntp, ws + P->o_X00), ++g_launches);
  return E2_OK;
}

// Integral blocks and row descriptors of the external classes.
void setup_classes(e2_problem* P, unsigned char* ws, cudaStream_t st) {
  const e2_desc& d = P->d;
  const int na = P->na, Lt = d.L_coulomb + d.L_extra;
  Ctx X = ctx(P, ws);
  const int modes[E2_NCLASS] = {-1, -1, INT_W02, -1, INT_W11, INT_W12, INT_W20, INT_W21, -1};
  const int cols[E2_NCLASS] = {0, 0, P->ntp, 0, 1 + na * na, na, P->ntp, na, 0};
  // factor columns for the blocks formed on the tensor pipe: <ab||tu>,
  // <ab||it> and <au||vw> as products over the factor index L
  const int64_t nva = (int64_t)P->nvc * na;
  double2* Yw = (double2*)(ws + P->o_vaY);
  double2* Zf = (double2*)(ws + P->o_vaZ);
  const bool on2 = P->M[2] > 0 && P->part_cnt[2] > 0, on5 = P->M[5] > 0 && P->part_cnt[5] > 0;
  const bool on1 = P->part_cnt[1] > 0;
  if ((on2 || on5 || on1) && nva > 0) {
    (k_vafactors<<<blocks(nva * Lt), 256, 0, st>>>(X.sp, X.Bo, X.wt, Lt, Yw, Zf), ++g_launches);
    (k_xfactors<<<blocks(((int64_t)P->nvc * P->ncc + (int64_t)na * na) * Lt), 256, 0, st>>>(
         X.sp, X.Bo, X.wt, Lt, (double2*)(ws + P->o_xYc), (double2*)(ws + P->o_xZaa)), ++g_launches);
  }
  for (int c = 0; c < E2_NCLASS; ++c) {
    if (modes[c] < 0 || P->M[c] == 0 || P->part_cnt[c] == 0) continue;
    (k_rows<<<blocks(P->M[c]), 256, 0, st>>>(c, X.sp, X.epsh, X.G, P->M[c], (RowInfo*)(ws + P->o_rows[c])), ++g_launches);
    if (c == 5) {
      // (ai|bt) = sum_L wt_L B_ai B_bt for all (a,i), (b,t), then <ab||it> = (ai|bt) - (at|bi)
      double2* X12 = (double2*)(ws + P->o_x12);
      zgemm(st, (int64_t)P->nvc * P->ncc, nva, Lt, (const double2*)(ws + P->o_xYc), Lt, 1, 0, Zf, nva, 1, 0, X12, nva, 1,
            0);
      (k_w12<<<blocks(P->M[c] * P->Kp[c]), 256, 0, st>>>(X.sp, X12, nva, P->M[c], P->Kp[c], (double2*)(ws + P->o_W[c])),
       ++g_launches);
      continue;
    }
    if (c == 2) {
      // (at|bu) = sum_L wt_L B_at B_bu on the tensor pipe, lower triangle
      // (a < b) in stripes of whole virtuals b, then <ab||tu> = (at|bu) - (au|bt)
      double2* Xv = (double2*)(ws + P->o_vaX);
      for (int b0 = 0, b1; b0 < P->nvc; b0 = b1) {
        b1 = b0 + 1;
        while (b1 < P->nvc && 16 * (size_t)(b1 + 1 - b0) * na * (size_t)(b1 + 1) * na <= P->va_cap) ++b1;
        const int64_t r0 = (int64_t)b0 * na, rows = (int64_t)(b1 - b0) * na, ldx = (int64_t)b1 * na;
        dim3 grid((unsigned)((rows + 63) / 64), (unsigned)((ldx + 63) / 64), 1);
        (k_zgemm64<<<grid, 256, 0, st>>>(rows, ldx, Lt, Yw + r0 * Lt, Lt, 1, 0, Zf, nva, 1, 0, Xv, ldx, 1, 0, Lt, 0,
                                          r0), ++g_launches);
        if (pairs(b1) > pairs(b0))
          (k_w02<<<blocks((pairs(b1) - pairs(b0)) * P->Kp[c]), 256, 0, st>>>(X.sp, Xv, ldx, b0, b1, P->Kp[c],
                                                                             (double2*)(ws + P->o_W[c])), ++g_launches);
      }
      continue;
    }
    (k_integrals<<<blocks(P->M[c] * P->Kp[c]), 256, 0, st>>>(modes[c], X.sp, X.Bo, X.wt, Lt, X.f, P->M[c], cols[c],
                                                             P->Kp[c], ws + P->o_W[c]), ++g_launches);
  }
  if (P->part_cnt[8] > 0)
    (k_integrals<<<blocks(P->ncp * P->nvp), 256, 0, st>>>(INT_G22, X.sp, X.Bo, X.wt, Lt, X.f, P->ncp, (int)P->nvp,
                                                         (int)P->nvp, ws + P->o_G22), ++g_launches);
  if (on1 && nva > 0) {  // (av|uw) for all (a,v), (u,w), then <au||vw> = (av|uw) - (aw|uv)
    double2* X01g = (double2*)(ws + P->o_x01);
    zgemm(st, nva, (int64_t)na * na, Lt, Yw, Lt, 1, 0, (const double2*)(ws + P->o_xZaa), (int64_t)na * na, 1, 0, X01g,
          (int64_t)na * na, 1, 0);
    (k_x01<<<blocks((int64_t)P->nvc * na * P->ntp), 256, 0, st>>>(X.sp, X01g, (double2*)(ws + P->o_X01)), ++g_launches);
  }
  if (P->part_cnt[3] > 0)
    (k_integrals<<<blocks((int64_t)P->ncc * P->ntp * na), 256, 0, st>>>(INT_X10, X.sp, X.Bo, X.wt, Lt, X.f, P->ncc,
                                                                       P->ntp * na, P->ntp * na, ws + P->o_X10), ++g_launches);
}


// Gamma_D of a column-tiled class in compacted form, GDc (+)= per tile
// W[:, klist]^T conj(T[:, perm]) over the chunk's Mc rows, split-K as zgemm.
void zgemm_gd_tiles(cudaStream_t st, const ColPlan& cp, const ColTiles& ctl, const double2* W, int Kp,
                    const double2* T, int64_t N, int64_t Mc, double2* GDc, int beta, int conjT = 1) {
  const int64_t czs = cp.krows * 64;
  const int nseg = splitk_segments(cp.gd_ctas, Mc, 16 * (size_t)czs);
  const int64_t kseg = (Mc + nseg - 1) / nseg;
  dim3 grid((unsigned)((cp.maxklen + 79) / 80), (unsigned)cp.tiles, (unsigned)nseg);
  if (nseg == 1) {
    (k_zgemm_gd_tiles<<<grid, 256, 0, st>>>(ctl, W, Kp, T, N, Mc, GDc, beta, kseg, 0, conjT), ++g_launches);
    return;
  }
  double2* part = (double2*)g_splitk;
  (k_zgemm_gd_tiles<<<grid, 256, 0, st>>>(ctl, W, Kp, T, N, Mc, part, 0, kseg, czs, conjT), ++g_launches);
  (k_zacc<<<blocks(czs), 256, 0, st>>>(part, nseg, czs, cp.krows, 64, GDc, 64, 1, beta), ++g_launches);
}

// Coupling tensors of root r, the active one- and two-particle blocks of
// its reference state, and E0 (Sec. 2.3).
void prepare_root(e2_problem* P, unsigned char* ws, cudaStream_t st, const double2* c, int r) {
  const int na = P->na;
  Ctx X = ctx(P, ws);
  Tabs T = tables(P, ws, r);
  const DevList L02 = dev_list(P, P->list_of[2], ws), L11 = dev_list(P, P->list_of[4], ws);
  build_tables(P, ws, st, c, T, true);
  const double2* Dcls[E2_NCLASS] = {nullptr, nullptr, T.DTU, nullptr, T.DTDU, T.DT, T.DTDUD, T.DTD, nullptr};
  for (int cls = 0; cls < E2_NCLASS; ++cls)
    if (P->use_cols[cls]) {
      const ColTiles ct = col_tiles(P, ws, r, cls);
      (k_dcompact<<<(unsigned)P->cplan[cls].tiles, 256, 0, st>>>(Dcls[cls], P->lists[P->list_of[cls]].n, ct,
                                                                 (double2*)ct.Dc), ++g_launches);
    }
  double2* g1 = (double2*)(ws + P->o_g1 + P->g_stride * r);
  double2* g2 = (double2*)(ws + P->o_g2 + P->g_stride * r);
  (k_gram<<<1 + na * na, 256, 0, st>>>(T.DTDU, T.DTDU, L11.n, 1 + na * na, g1), ++g_launches);
  if (P->ntp > 0 && L02.n > 0) (k_gram<<<P->ntp * P->ntp, 256, 0, st>>>(T.DTU, T.DTU, L02.n, P->ntp, g2), ++g_launches);
  else cudaMemsetAsync(g2, 0, 16 * (size_t)std::max(P->ntp * P->ntp, 1), st);
  (k_e0<<<1, 256, 0, st>>>(g1, g2, X.f, (const double2*)(ws + P->o_X00), X.sp, P->ntp, X.EO, X.E0p + r, X.E0d + r),
   ++g_launches);
}

// Classes (2,2), (0,1), (1,0), (0,0) of root r (their partial slots).
template <class Mark>
void launch_sparse_classes(e2_problem* P, unsigned char* ws, cudaStream_t st, int r, const double2* c, Mark mark) {
  Ctx X = ctx(P, ws);
  Tabs T = tables(P, ws, r);
  DevList Lc[E2_NCLASS];
  for (int k = 0; k < E2_NCLASS; ++k) Lc[k] = dev_list(P, P->list_of[k], ws);
  const double b = P->d.level_shift_b;
  double* part = (double*)(ws + P->o_part);
  auto poff = [&](int cls) { return part + P->part_off[r * E2_NCLASS + cls]; };
  if (P->part_cnt[8] > 0) {
    const DevList& L = Lc[8];
    dim3 grid(blocks(L.n), (unsigned)(P->nvb * (P->nvb + 1) / 2), (unsigned)P->ncp);
    mark(8, 0);
    (k_class22<<<grid, 256, 0, st>>>(L, X.sp, c, (const double*)(ws + P->o_G22), X.epsh, X.G, X.E0p + r, b, P->nvb,
                                    poff(8)), ++g_launches);
    mark(8, 1);
  }
  if (P->part_cnt[1] > 0) {
    dim3 grid(blocks(Lc[1].n), (unsigned)P->nvc);
    mark(1, 0);
    (k_class01<<<grid, 256, 0, st>>>(Lc[1], Lc[5], Lc[2], P->das, X.sp, X.binom, T.DT, T.DTU,
                                    (const double2*)(ws + P->o_X01), X.f, X.epsh, X.E0p + r, b, poff(1)), ++g_launches);
    mark(1, 1);
  }
  if (P->part_cnt[3] > 0) {
    dim3 grid(blocks(Lc[3].n), (unsigned)P->ncc);
    mark(3, 0);
    (k_class10<<<grid, 256, 0, st>>>(Lc[3], Lc[7], Lc[5], P->das, X.sp, X.binom, T.DTD, T.DT,
                                    (const double2*)(ws + P->o_X10), X.f, X.epsh, X.E0p + r, b, poff(3)), ++g_launches);
    mark(3, 1);
  }
  if (P->part_cnt[0] > 0) {
    mark(0, 0);
    (k_class00<<<blocks(Lc[0].n), 256, 0, st>>>(Lc[0], Lc[4], Lc[2], P->das, X.sp, X.binom, T.DTDU, T.DTU,
                                               (const double2*)(ws + P->o_X00), X.f, X.E0p + r, b, poff(0)), ++g_launches);
    mark(0, 1);
  }
}

// E2_class and E2 of every root from the partial slots (fixed order).
void launch_reduce(e2_problem* P, unsigned char* ws, cudaStream_t st, double* E2, double* E2_class, double* E0) {
  const int R = P->d.n_roots;
  double* e2c = E2_class ? E2_class : (double*)(ws + P->o_e2c);
  (k_reduce<<<R * E2_NCLASS, 256, 0, st>>>((const double*)(ws + P->o_part), (const int64_t*)(ws + P->o_partoff),
                                           (const int64_t*)(ws + P->o_partcnt), (const double2*)(ws + P->o_g1),
                                           (int)(P->g_stride / 16), R, e2c), ++g_launches);
  (k_finalize<<<1, 32, 0, st>>>(e2c, R, E2, (const double*)(ws + P->o_E0), E0), ++g_launches);
}

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
  cudaGetLastError();
  g_launches = 0;
  if (setup_common(P, in, ws, st) != E2_OK) return E2_ERR_CUDA;
  setup_classes(P, ws, st);
  const e2_desc& d = P->d;
  const int R = d.n_roots;
  const double b = d.level_shift_b;
  Ctx X = ctx(P, ws);
  const DevList LP = dev_list(P, P->listP, ws);
  DevList Lc[E2_NCLASS];
  for (int c = 0; c < E2_NCLASS; ++c) Lc[c] = dev_list(P, P->list_of[c], ws);
  double* part = (double*)(ws + P->o_part);
  for (int r = 0; r < R; ++r) {
    const double2* c = (const double2*)in->c + (int64_t)r * LP.n;
    Tabs T = tables(P, ws, r);
    prepare_root(P, ws, st, c, r);

    auto poff = [&](int cls) { return part + P->part_off[r * E2_NCLASS + cls]; };
    const double2* Dfor[E2_NCLASS] = {nullptr, nullptr, T.DTU, nullptr, T.DTDU, T.DT, T.DTDUD, T.DTD, nullptr};
    auto mark = [&](int cls, int k) {
      if (P->prof_on && r == 0) cudaEventRecord(P->prof[2 * cls + k], st);
    };
    for (int cls : {2, 5, 7, 4, 6}) {
      if (P->part_cnt[cls] == 0) continue;
      const DevList& L = Lc[cls];
      dim3 grid((unsigned)((P->M[cls] + 63) / 64), (unsigned)((L.n + 63) / 64));
      mark(cls, 0);
      (k_class_gemm<<<grid, 256, 0, st>>>((const double2*)(ws + P->o_W[cls]), Dfor[cls], P->M[cls], L.n, P->Kp[cls],
                                         (const RowInfo*)(ws + P->o_rows[cls]), L.U, L.eA, X.E0p + r, b, poff(cls), AdjOut{},
                                         col_tiles(P, ws, r, cls)), ++g_launches);
      mark(cls, 1);
    }
    launch_sparse_classes(P, ws, st, r, c, mark);
  }
  double* e2c = E2_class ? E2_class : (double*)(ws + P->o_e2c);
  (k_reduce<<<R * E2_NCLASS, 256, 0, st>>>(part, (const int64_t*)(ws + P->o_partoff), (const int64_t*)(ws + P->o_partcnt),
                                          (const double2*)(ws + P->o_g1), (int)(P->g_stride / 16), R, e2c), ++g_launches);
  (k_finalize<<<1, 32, 0, st>>>(e2c, R, E2, X.E0d, E0), ++g_launches);
  P->launches = g_launches;
  if (cudaGetLastError() != cudaSuccess) return E2_ERR_CUDA;
  return E2_OK;
}

e2_status e2_partials(const e2_problem* P, const void* workspace, int root, int cls, const double** partials,
                      int64_t* count, int64_t* row_tiles, const int32_t** columns) {
  if (!P || !workspace || !partials || !count) return E2_ERR_INVALID_ARG;
  if (root < 0 || root >= P->d.n_roots || cls < 0 || cls >= E2_NCLASS) return E2_ERR_INVALID_ARG;
  *partials = (const double*)((const unsigned char*)workspace + P->o_part) + P->part_off[root * E2_NCLASS + cls];
  *count = P->part_cnt[cls];
  const bool dense = cls == 2 || cls == 5 || cls == 7 || cls == 4 || cls == 6;
  if (row_tiles) *row_tiles = dense ? (P->M[cls] + 63) / 64 : 0;
  if (columns)
    *columns = P->use_cols[cls] ? (const int32_t*)((const unsigned char*)workspace + P->cplan[cls].o_perm) : nullptr;
  return E2_OK;
}

e2_status e2_class_tiles(const e2_problem* P, int cls, int64_t* tiles, int64_t* krows, int* in_use) {
  if (!P || cls < 0 || cls >= E2_NCLASS) return E2_ERR_INVALID_ARG;
  const ColPlan& cp = P->cplan[cls];
  if (tiles) *tiles = cp.built ? cp.tiles : 0;
  if (krows) *krows = cp.built ? cp.krows : 0;
  if (in_use) *in_use = P->use_cols[cls] ? 1 : 0;
  return E2_OK;
}

e2_status e2_class_tiles_copy(const e2_problem* P, int cls, int32_t* perm, int32_t* tdesc, int32_t* klist) {
  if (!P || cls < 0 || cls >= E2_NCLASS || !perm || !tdesc || !klist) return E2_ERR_INVALID_ARG;
  const ColPlan& cp = P->cplan[cls];
  if (!cp.built) return E2_ERR_UNSUPPORTED;
  std::copy(cp.perm.begin(), cp.perm.end(), perm);
  std::copy(cp.tdesc.begin(), cp.tdesc.end(), tdesc);
  std::copy(cp.klist.begin(), cp.klist.end(), klist);
  return E2_OK;
}

e2_status e2_set_class_tiles(e2_problem* P, int cls, int on) {
  if (!P || cls < 0 || cls >= E2_NCLASS) return E2_ERR_INVALID_ARG;
  if (on && !P->cplan[cls].built) return E2_ERR_UNSUPPORTED;
  P->use_cols[cls] = on != 0;
  return E2_OK;
}

e2_status e2_autotune(e2_problem* P, const e2_inputs* in, void* workspace, size_t workspace_bytes, void* stream_,
                      float* ms_out) {
  if (!P || !in || !in->h || !in->B_c || !in->c) return E2_ERR_INVALID_ARG;
  if (P->d.L_extra > 0 && (!in->B_x || !in->w_x)) return E2_ERR_INVALID_ARG;
  if (!std::isfinite(in->lambda)) return E2_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < P->ws_bytes || ((uintptr_t)workspace & 255)) return E2_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream_;
  unsigned char* ws = (unsigned char*)workspace;
  cudaGetLastError();
  if (setup_common(P, in, ws, st) != E2_OK) return E2_ERR_CUDA;
  setup_classes(P, ws, st);
  bool cand[E2_NCLASS];
  for (int c = 0; c < E2_NCLASS; ++c) {
    cand[c] = P->cplan[c].built && P->part_cnt[c] > 0;
    if (cand[c]) P->use_cols[c] = true;  // so that root 0's compacted tables are built
  }
  prepare_root(P, ws, st, (const double2*)in->c, 0);
  Ctx X = ctx(P, ws);
  Tabs T = tables(P, ws, 0);
  const double2* Dfor[E2_NCLASS] = {nullptr, nullptr, T.DTU, nullptr, T.DTDU, T.DT, T.DTDUD, T.DTD, nullptr};
  double* part = (double*)(ws + P->o_part);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return E2_ERR_CUDA;
  for (int c = 0; c < E2_NCLASS; ++c) {
    if (ms_out) ms_out[2 * c] = ms_out[2 * c + 1] = 0.f;
    if (!cand[c]) continue;
    const DevList L = dev_list(P, P->list_of[c], ws);
    dim3 grid((unsigned)((P->M[c] + 63) / 64), (unsigned)((L.n + 63) / 64));
    float t[2] = {0.f, 0.f};
    for (int v = 0; v < 2; ++v) {  // v = 0: plain columns, 1: compacted column tiles
      P->use_cols[c] = v == 1;
      auto launch = [&] {
        k_class_gemm<<<grid, 256, 0, st>>>((const double2*)(ws + P->o_W[c]), Dfor[c], P->M[c], L.n, P->Kp[c],
                                           (const RowInfo*)(ws + P->o_rows[c]), L.U, L.eA, X.E0p, P->d.level_shift_b,
                                           part + P->part_off[c], AdjOut{}, col_tiles(P, ws, 0, c));
      };
      launch();
      cudaEventRecord(e0, st);
      for (int k = 0; k < 2; ++k) launch();
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&t[v], e0, e1);
    }
    P->use_cols[c] = t[1] < t[0];
    if (ms_out) {
      ms_out[2 * c] = 0.5f * t[0];
      ms_out[2 * c + 1] = 0.5f * t[1];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return cudaGetLastError() == cudaSuccess ? E2_OK : E2_ERR_CUDA;
}

e2_status e2_launch_count(const e2_problem* P, int64_t* n) {
  if (!P || !n) return E2_ERR_INVALID_ARG;
  *n = P->launches;
  return E2_OK;
}

e2_status e2_profile_events(e2_problem* P, void* const* events) {
  if (!P) return E2_ERR_INVALID_ARG;
  P->prof_on = events != nullptr;
  if (events)
    for (int k = 0; k < 2 * E2_NCLASS; ++k) P->prof[k] = (cudaEvent_t)events[k];
  return E2_OK;
}

e2_status e2_fp64_peak(void* workspace, size_t workspace_bytes, void* stream_, double* dmma_tflops,
                       double* dfma_tflops) {
  if (!dmma_tflops || !dfma_tflops) return E2_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int nb = sms * 8, nt = 256;
  if (!workspace || workspace_bytes < sizeof(double) * nb * nt) return E2_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream_;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return E2_ERR_CUDA;
  double* out = (double*)workspace;
  const int iters = 2048;
  float ms = 0.f;
  (k_peak_dmma<<<nb, nt, 0, st>>>(out, iters), ++g_launches);
  cudaEventRecord(e0, st);
  for (int k = 0; k < 3; ++k) (k_peak_dmma<<<nb, nt, 0, st>>>(out, iters), ++g_launches);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *dmma_tflops = 3.0 * (double)nb * (nt / 32) * iters * 4 * (16.0 * 8 * 8 * 2) / (ms * 1e-3) / 1e12;
  (k_peak_dfma<<<nb, nt, 0, st>>>(out, iters), ++g_launches);
  cudaEventRecord(e0, st);
  for (int k = 0; k < 3; ++k) (k_peak_dfma<<<nb, nt, 0, st>>>(out, iters), ++g_launches);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  *dfma_tflops = 3.0 * (double)nb * nt * iters * 8 * 2.0 / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return cudaGetLastError() == cudaSuccess ? E2_OK : E2_ERR_CUDA;
}


// ------------------------------------------------------------------ batches

struct e2_batch {
  std::vector<e2_problem*> jobs;
  std::vector<size_t> off;          // workspace offset of each job's forward layout
  size_t o_jobs = 0, o_items = 0, o_counter = 0, bytes = 0;
  std::vector<GemmJob> gj;          // absolute pointers, built by e2_batch_prepare
  std::vector<WorkItem> items;
  int64_t n_items = 0;
  const void* prepared = nullptr;
  int64_t launches = 0;
};

e2_status e2_batch_create(e2_problem* const* jobs, int n_jobs, e2_batch** out) {
  if (!out) return E2_ERR_INVALID_ARG;
  *out = nullptr;
  if (!jobs || n_jobs < 1) return E2_ERR_INVALID_ARG;
  e2_batch* B = new (std::nothrow) e2_batch();
  if (!B) return E2_ERR_INVALID_ARG;
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
      if (jobs[j]->part_cnt[c] > 0) {
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
      if (P->part_cnt[c] == 0) continue;
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
    for (int r = 0; r < P->d.n_roots; ++r)
      launch_sparse_classes(P, w, st, r, (const double2*)inputs[j].c + (int64_t)r * P->lists[P->listP].n, nomark);
    launch_reduce(P, w, st, E2[j], E2_class ? E2_class[j] : nullptr, nullptr);
  }
  B->launches = g_launches;
  if (cudaGetLastError() != cudaSuccess) return E2_ERR_CUDA;
  return E2_OK;
}

e2_status e2_batch_launch_count(const e2_batch* B, int64_t* n) {
  if (!B || !n) return E2_ERR_INVALID_ARG;
  *n = B->launches;
  return E2_OK;
}

e2_status e2_backward_workspace_size(const e2_problem* P, size_t* bytes) {
  if (!P || !bytes) return E2_ERR_INVALID_ARG;
  *bytes = P->bwd_bytes;
  return E2_OK;
}

e2_status e2_backward(e2_problem* P, const e2_inputs* in, const double* seed, void* workspace, size_t workspace_bytes,
                      void* stream_, double* g_h, double* g_c, double* g_Bc, double* g_Bx, double* dE2_dlambda,
                      double* E2) {
  if (!P || !in || !seed || !in->h || !in->B_c || !in->c) return E2_ERR_INVALID_ARG;
  if (P->d.L_extra > 0 && (!in->B_x || !in->w_x)) return E2_ERR_INVALID_ARG;
  if (!std::isfinite(in->lambda)) return E2_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < P->bwd_bytes || ((uintptr_t)workspace & 255)) return E2_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream_;
  unsigned char* ws = (unsigned char*)workspace;
  const e2_desc& d = P->d;
  const int R = d.n_roots, na = P->na;
  const double b = d.level_shift_b;
  cudaGetLastError();
  g_launches = 0;
  if (setup_common(P, in, ws, st) != E2_OK) return E2_ERR_CUDA;
  setup_classes(P, ws, st);
  struct SplitScope {  // split-K scratch of this pass's GEMM helpers
    SplitScope(void* p, size_t n) { g_splitk = p; g_splitk_bytes = n; }
    ~SplitScope() { g_splitk = nullptr; g_splitk_bytes = 0; }
  } split_scope(ws + P->o_bPart, P->bpart_bytes);
  Ctx X = ctx(P, ws);
  const DevList LP = dev_list(P, P->listP, ws);
  DevList Lc[E2_NCLASS];
  for (int c = 0; c < E2_NCLASS; ++c) Lc[c] = dev_list(P, P->list_of[c], ws);
  auto B = [&](size_t o) { return (void*)(ws + o); };
  double2* Gf = (double2*)B(P->o_bGf);
  double* Nx = (double*)B(P->o_bNx);
  double* Nt = (double*)B(P->o_bNt);
  double* Nd = (double*)B(P->o_bNd);
  double* scal = (double*)B(P->o_bScal);
  double2* Gc = (double2*)B(P->o_bGc);
  double2* sig = (double2*)B(P->o_bSig);
  cudaMemsetAsync(Gf, 0, 16 * (size_t)P->n * P->nocc, st);
  cudaMemsetAsync(Nx, 0, 8 * (size_t)(P->nx + 1), st);
  cudaMemsetAsync(Nt, 0, 8 * (size_t)std::max(na, 1), st);
  const bool want_B = g_Bc || g_Bx || dE2_dlambda;
  const int nx = P->nx;
  const int64_t npair = P->npair;
  double* Ge = (double*)B(P->o_bGe);
  double* Gea = (double*)B(P->o_bGea);
  double* Ntt = (double*)B(P->o_bNtt);
  double2* Gt = (double2*)B(P->o_bGt);
  double* Hocc = (double*)B(P->o_bHocc);
  double* Zm = (double*)B(P->o_bZ);
  double* Zs = (double*)B(P->o_bZs);
  if (want_B) {
    cudaMemsetAsync(Ge, 0, 8 * (size_t)std::max(nx, 1) * std::max(nx, 1), st);
    cudaMemsetAsync(Gea, 0, 8 * (size_t)std::max(nx, 1) * std::max(na, 1), st);
    cudaMemsetAsync(Ntt, 0, 8 * (size_t)na * na, st);
    cudaMemsetAsync(Gt, 0, 16 * (size_t)npair * npair, st);
  }
  // denominators of rows with external indices: Ge += Z^T diag(hsum) Z, Gea += Z^T Hocc
  auto zpair = [&](const RowInfo* rows, int64_t M, const double* hs, const double* hocc) {
    (k_zmat<<<blocks(M * nx), 256, 0, st>>>(rows, M, nx, Zm), ++g_launches);
    (k_zscale<<<blocks(M * nx), 256, 0, st>>>(Zm, hs, M, nx, Zs), ++g_launches);
    dgemm(st, nx, nx, M, Zm, 1, nx, Zs, nx, 1, Ge, nx, 1);
    dgemm(st, nx, na, M, Zm, 1, nx, hocc, na, 1, Gea, na, 1);
  };
  const bool on[E2_NCLASS] = {P->part_cnt[0] > 0, P->part_cnt[1] > 0, P->part_cnt[2] > 0, P->part_cnt[3] > 0,
                              P->part_cnt[4] > 0, P->part_cnt[5] > 0, P->part_cnt[6] > 0, P->part_cnt[7] > 0,
                              P->part_cnt[8] > 0};
  for (int r = 0; r < R; ++r) {
    const double2* c = (const double2*)in->c + (int64_t)r * LP.n;
    prepare_root(P, ws, st, c, r);
    const double s = seed[r];
    double* part_r = (double*)(ws + P->o_part);
    auto poff = [&](int cls) { return E2 ? part_r + P->part_off[r * E2_NCLASS + cls] : nullptr; };
    auto nomark = [](int, int) {};
    if (s == 0.0) {
      if (E2) launch_sparse_classes(P, ws, st, r, c, nomark);
      if (g_c) cudaMemsetAsync(g_c + 2 * (size_t)r * LP.n, 0, 16 * (size_t)LP.n, st);
      if (E2) {  // no amplitudes for this root: the forward's dense classes alone
        Tabs T0 = tables(P, ws, r);
        const double2* Df[E2_NCLASS] = {nullptr, nullptr, T0.DTU, nullptr, T0.DTDU, T0.DT, T0.DTDUD, T0.DTD, nullptr};
        for (int cls : {2, 5, 7, 4, 6}) {
          if (!on[cls]) continue;
          dim3 grid((unsigned)((P->M[cls] + 63) / 64), (unsigned)((Lc[cls].n + 63) / 64));
          (k_class_gemm<<<grid, 256, 0, st>>>((const double2*)(ws + P->o_W[cls]), Df[cls], P->M[cls], Lc[cls].n,
                                              P->Kp[cls], (const RowInfo*)(ws + P->o_rows[cls]), Lc[cls].U, Lc[cls].eA,
                                              X.E0p + r, b, poff(cls), AdjOut{}, col_tiles(P, ws, r, cls)), ++g_launches);
        }
      }
      continue;
    }
    Tabs T = tables(P, ws, r);
    Tabs GT{(double2*)(ws + P->o_gD + (P->o_DT - P->o_dstart)), (double2*)(ws + P->o_gD + (P->o_DTD - P->o_dstart)),
            (double2*)(ws + P->o_gD + (P->o_DTU - P->o_dstart)), (double2*)(ws + P->o_gD + (P->o_DTDUD - P->o_dstart)),
            (double2*)(ws + P->o_gD + (P->o_DTDU - P->o_dstart))};
    const double2* g1 = (const double2*)(ws + P->o_g1 + P->g_stride * r);
    cudaMemsetAsync(ws + P->o_gD, 0, P->d_stride, st);
    cudaMemsetAsync(Gc, 0, 16 * (size_t)LP.n, st);
    cudaMemsetAsync(scal, 0, 16, st);
    if (want_B) cudaMemsetAsync(B(P->o_bGX00), 0, 16 * (size_t)std::max(P->ntp * P->ntp, 1), st);
    double* hsum = (double*)B(P->o_bHsum);
    double* hA = (double*)B(P->o_bHA);
    // dense classes: amplitudes in row chunks, Gamma_D += W^T conj(T)
    const double2* Dfor[E2_NCLASS] = {nullptr, nullptr, T.DTU, nullptr, T.DTDU, T.DT, T.DTDUD, T.DTD, nullptr};
    double2* GDfor[E2_NCLASS] = {nullptr, nullptr, GT.DTU, nullptr, GT.DTDU, GT.DT, GT.DTDUD, GT.DTD, nullptr};
    for (int cls : {2, 5, 7, 4, 6}) {
      if (!on[cls]) continue;
      const DevList& L = Lc[cls];
      const int64_t M = P->M[cls], N = L.n, Kp = P->Kp[cls];
      const int64_t rt = (M + 63) / 64, ct = (N + 63) / 64;
      const double2* W = (const double2*)(ws + P->o_W[cls]);
      // the class kernel reads the column tiles whenever the class uses them;
      // the Gamma products do so for the 8-granular plans (a 16-row table
      // gains nothing at the products' 8-wide output granularity)
      const bool tiled = P->use_cols[cls] && P->cplan[cls].gran == 8;
      const ColPlan& cp = P->cplan[cls];
      const ColTiles ctl = col_tiles(P, ws, r, cls);
      for (int64_t m0 = 0; m0 < M; m0 += P->chunk_rows[cls]) {
        const int64_t Mc = std::min<int64_t>(P->chunk_rows[cls], M - m0);
        AdjOut adj{(double2*)B(P->o_bT), want_B ? (double*)B(P->o_bHm) : nullptr, (double*)B(P->o_bHrow),
                   (double*)B(P->o_bHcol), (double*)B(P->o_bScalT), m0, Mc, s, g1, poff(cls), rt};
        dim3 grid((unsigned)((Mc + 63) / 64), (unsigned)ct);
        (k_class_gemm<<<grid, 256, 0, st>>>(W, Dfor[cls], M, N, (int)Kp, (const RowInfo*)(ws + P->o_rows[cls]), L.U,
                                            L.eA, X.E0p + r, b, nullptr, adj, col_tiles(P, ws, r, cls)), ++g_launches);
        // Gamma_D[x][A] += sum_e W[e][x] conj(T[e][A]) (split over the rows of the chunk)
        if (tiled)
          zgemm_gd_tiles(st, cp, ctl, W + m0 * Kp, (int)Kp, adj.T, N, Mc, (double2*)B(P->o_bGDc), m0 > 0);
        else if (Kp >= 64)
          zgemm(st, Kp, N, Mc, W + m0 * Kp, 1, Kp, 0, adj.T, N, 1, 1, GDfor[cls], N, 1, 1, 64);
        else
          zgemm(st, N, Kp, Mc, adj.T, 1, N, 1, W + m0 * Kp, Kp, 1, 0, GDfor[cls], 1, N, 1, 16);
        if (cls == 4)
          (k_rowdot<<<(unsigned)Mc, 256, 0, st>>>(adj.T, T.DTDU, N, (double2*)B(P->o_bRowdot) + m0), ++g_launches);
        if (want_B) {  // Gamma_W = conj(T) D^T and the per-row occupation sums of eta
          double2* GW = (double2*)B(P->o_bGW[cls]) + m0 * Kp;
          if (tiled) {  // per tile over its compacted rows, then summed per table row in tile order
            dim3 g((unsigned)((Mc + 63) / 64), (unsigned)((cp.maxklen + 79) / 80), (unsigned)cp.tiles);
            (k_zgemm_gw_tiles<<<g, 256, 0, st>>>(ctl, adj.T, N, Mc, cp.krows, (double2*)B(P->o_bGWc), 1),
             ++g_launches);
            (k_gw_reduce<<<blocks(Mc * Kp), 256, 0, st>>>(ctl.tdesc, (const int32_t*)(ws + cp.o_pos), cp.tiles,
                                                         (int)Kp, (const double2*)B(P->o_bGWc), cp.krows, Mc, GW,
                                                         (int)Kp, Kp), ++g_launches);
          } else {
            zgemm(st, Mc, Kp, N, adj.T, N, 1, 1, Dfor[cls], 1, N, 0, GW, Kp, 1, 0, Kp >= 64 ? 64 : 16);
          }
          (k_hocc<<<(unsigned)Mc, 256, 0, st>>>(adj.Hm, L, na, Hocc + m0 * na), ++g_launches);
        }
      }
      if (tiled)
        (k_gd_scatter<<<(unsigned)cp.tiles, 256, 0, st>>>(ctl, (const double2*)B(P->o_bGDc), N, GDfor[cls]),
         ++g_launches);
      if (cls == 4) (k_fock11<<<blocks(M), 256, 0, st>>>((const double2*)B(P->o_bRowdot), X.sp, Gf), ++g_launches);
      (k_rowsum<<<blocks(M), 256, 0, st>>>((const double*)B(P->o_bHrow), M, ct, 0, hsum), ++g_launches);
      (k_xmarg<<<P->nx, 256, 0, st>>>((const RowInfo*)(ws + P->o_rows[cls]), hsum, M, P->nx, Nx), ++g_launches);
      (k_colsum<<<blocks(N), 256, 0, st>>>((const double*)B(P->o_bHcol), rt, N, 0, hA), ++g_launches);
      (k_amarg<<<na, 256, 0, st>>>(L, hA, Nt), ++g_launches);
      (k_scalsum<<<1, 256, 0, st>>>((const double*)B(P->o_bScalT), rt * ct, scal), ++g_launches);
      if (want_B) {
        zpair((const RowInfo*)(ws + P->o_rows[cls]), M, hsum, Hocc);
        (k_ntt<<<na * na, 256, 0, st>>>(L, hA, na, Ntt), ++g_launches);
        const int modes[E2_NCLASS] = {-1, -1, INT_W02, -1, INT_W11, INT_W12, INT_W20, INT_W21, -1};
        const int cols[E2_NCLASS] = {0, 0, P->ntp, 0, 1 + na * na, na, P->ntp, na, 0};
        (k_gint<<<blocks(M * cols[cls]), 256, 0, st>>>(modes[cls], X.sp, (const double2*)B(P->o_bGW[cls]), M, cols[cls],
                                                       (int)Kp, Gt, npair), ++g_launches);
      }
    }
    // class (2,2)
    double* c22 = nullptr;
    if (on[8]) {
      const DevList& L = Lc[8];
      const int64_t nyb = (int64_t)P->nvb * (P->nvb + 1) / 2, yz = nyb * P->ncp;
      dim3 grid(blocks(L.n), (unsigned)nyb, (unsigned)P->ncp);
      (k_class22_bwd<<<grid, 256, 0, st>>>(L, X.sp, c, (const double*)(ws + P->o_G22), X.epsh, X.G, X.E0p + r, b,
                                           P->nvb, s, g1, (double*)B(P->o_bC22p), (double*)B(P->o_bH22p),
                                           (double*)B(P->o_bV22), poff(8)), ++g_launches);
      c22 = (double*)B(P->o_bC22);
      (k_colsum<<<blocks(L.n), 256, 0, st>>>((const double*)B(P->o_bC22p), yz, L.n, 0, c22), ++g_launches);
      (k_colsum<<<blocks(L.n), 256, 0, st>>>((const double*)B(P->o_bH22p), yz, L.n, 0, hA), ++g_launches);
      (k_amarg<<<na, 256, 0, st>>>(L, hA, Nt), ++g_launches);
      (k_class22_marg<<<(unsigned)(P->nvc + P->ncc + 1), 256, 0, st>>>((const double*)B(P->o_bV22), (int)blocks(L.n),
                                                                   P->nvb, P->ncp, X.sp, Nx, scal), ++g_launches);
      if (want_B) {
        const int64_t M22 = P->ncp * P->nvp;
        double* hs22 = (double*)B(P->o_bHs22);
        double* P22 = (double*)B(P->o_bP22);
        (k_class22_rows<<<(unsigned)M22, 256, 0, st>>>(L, X.sp, c, (const double*)(ws + P->o_G22), X.epsh, X.G,
                                                       X.E0p + r, b, s, g1, hs22, Hocc, P22), ++g_launches);
        (k_rows<<<blocks(M22), 256, 0, st>>>(8, X.sp, X.epsh, X.G, M22, (RowInfo*)B(P->o_bR22)), ++g_launches);
        zpair((const RowInfo*)B(P->o_bR22), M22, hs22, Hocc);
        (k_ntt<<<na * na, 256, 0, st>>>(L, hA, na, Ntt), ++g_launches);
        const int Lt = d.L_coulomb + d.L_extra;
        (k_integrals<<<blocks(M22), 256, 0, st>>>(INT_G22C, X.sp, X.Bo, X.wt, Lt, X.f, P->ncp, (int)P->nvp,
                                                  (int)P->nvp, B(P->o_bG22c)), ++g_launches);
        (k_g22coef<<<blocks(M22), 256, 0, st>>>((const double2*)B(P->o_bG22c), P22, M22, (double2*)B(P->o_bGg22)),
         ++g_launches);
        (k_gint<<<blocks(M22), 256, 0, st>>>(INT_G22C, X.sp, (const double2*)B(P->o_bGg22), P->ncp, (int)P->nvp,
                                             (int)P->nvp, Gt, npair), ++g_launches);
      }
    }
    // gather classes
    for (int cls : {1, 3, 0}) {
      if (!on[cls]) continue;
      const DevList& L = Lc[cls];
      const int nrow = (int)P->M[cls];
      double2* Tg = (double2*)B(P->o_bGT);
      double* Hg = (double*)B(P->o_bGH);
      double* GVg = (double*)B(P->o_bGV);
      dim3 grid(blocks(L.n), (unsigned)nrow);
      (k_gather_t<<<grid, 256, 0, st>>>(cls, L, Lc[5], Lc[2], Lc[7], Lc[4], P->das, X.sp, X.binom, T.DT, T.DTU, T.DTD,
                                        T.DTDU, (const double2*)(ws + P->o_X01), (const double2*)(ws + P->o_X10),
                                        (const double2*)(ws + P->o_X00), X.f, X.epsh, X.E0p + r, b, s, g1, Tg, Hg,
                                        GVg, poff(cls)), ++g_launches);
      (k_sum2<<<1, 256, 0, st>>>(Hg, GVg, (int64_t)nrow * L.n, scal), ++g_launches);
      if (cls == 1) (k_rowsum_wide<<<(unsigned)nrow, 256, 0, st>>>(Hg, L.n, 1, Nx + P->ncc), ++g_launches);
      if (cls == 3) (k_rowsum_wide<<<(unsigned)nrow, 256, 0, st>>>(Hg, L.n, 1, Nx), ++g_launches);
      (k_colsum<<<blocks(L.n), 256, 0, st>>>(Hg, nrow, L.n, 0, hA), ++g_launches);
      (k_amarg<<<na, 256, 0, st>>>(L, hA, Nt), ++g_launches);
      // one-body parts: Gamma_f and the D^t / D^{t+} / D^{t+u} coefficients
      const int nk = (cls == 0) ? na * na : na;
      const DevList& Lsrc = (cls == 1) ? Lc[5] : (cls == 3) ? Lc[7] : Lc[4];
      const double2* Dsrc = (cls == 1) ? T.DT : (cls == 3) ? T.DTD : T.DTDU;
      double2* GDsrc = (cls == 1) ? GT.DT : (cls == 3) ? GT.DTD : GT.DTDU;
      if (Lsrc.n > 0) {
        (k_gather_fock<<<dim3(nk, nrow), 256, 0, st>>>(cls, L, Lsrc, P->das, X.sp, X.binom, Dsrc, Tg, Gf), ++g_launches);
        (k_gather_d1<<<blocks(Lsrc.n), 256, 0, st>>>(cls, L, Lsrc, P->das, X.sp, X.binom, Tg, nrow, X.f, GDsrc),
         ++g_launches);
      }
      // two-body parts: per removed spinor u (or pair t<u) the shifted
      // amplitudes Tsh[row][B] = conj(t[row][B + ...]) * sign give
      //   Gamma_D[x][B] += sum_row X[row][...][x] Tsh[row][B]        (reference gradient)
      //   Gamma_X[row][...][x] = sum_B Tsh[row][B] D[x][B]            (integral coefficients)
      if (want_B) {
        (k_rowsum_wide<<<(unsigned)nrow, 256, 0, st>>>(Hg, L.n, 0, hsum), ++g_launches);
        (k_hocc<<<(unsigned)nrow, 256, 0, st>>>(Hg, L, na, Hocc), ++g_launches);
        if (cls != 0) {
          (k_rows<<<blocks(nrow), 256, 0, st>>>(cls, X.sp, X.epsh, X.G, nrow, (RowInfo*)B(P->o_bRg)), ++g_launches);
          zpair((const RowInfo*)B(P->o_bRg), nrow, hsum, Hocc);
        }
        (k_ntt<<<na * na, 256, 0, st>>>(L, hA, na, Ntt), ++g_launches);
      }
      double2* Tsh = (double2*)B(P->o_bTsh);
      const int ntp = P->ntp;
      // Gamma_D[x][B] += sum_(row,s) X[row][s][x] Tsh[(row,s)][B] and
      // Gamma_X[row][s][x] = sum_B Tsh[(row,s)][B] D[x][B], rows in chunks that fit Tsh
      // With the (0,2) list's column tiles in use, the products that meet
      // D^{tu} run over the tiles' compacted rows (tcls = 2).
      auto shifted = [&](const DevList& Ltab, int S, int pairs_mode, int nx_, const double2* Xint, const double2* D,
                         double2* GD, double2* GX, int gx_beta, int bn, int tcls) {
        const int64_t nb = Ltab.n;
        if (nb == 0 || S == 0) return;
        const bool tl = tcls >= 0 && P->use_cols[tcls];
        const ColPlan& cpt = P->cplan[tcls >= 0 ? tcls : 0];
        const ColTiles ctt = tl ? col_tiles(P, ws, r, tcls) : ColTiles{nullptr, nullptr, nullptr, nullptr};
        int64_t rcap = (int64_t)(P->tsh_bytes / (16 * (size_t)S * nb));
        if (tl && want_B) rcap = std::min<int64_t>(rcap, (int64_t)(P->gwc_bytes / (16 * (size_t)S * cpt.krows)));
        const int rc = (int)std::max<int64_t>(1, std::min<int64_t>(nrow, rcap));
        for (int r0 = 0; r0 < nrow; r0 += rc) {
          const int nr = std::min(rc, nrow - r0);
          (k_tshift<<<dim3(blocks(nb), nr, S), 256, 0, st>>>(L, Ltab, P->das, X.binom, Tg, r0, pairs_mode, Tsh),
           ++g_launches);
          const int64_t k = (int64_t)nr * S;
          const double2* Xr = Xint + (int64_t)r0 * S * nx_;
          if (tl)
            zgemm_gd_tiles(st, cpt, ctt, Xr, nx_, Tsh, nb, k, (double2*)B(P->o_bGDc), r0 > 0, 0);
          else
            zgemm(st, nx_, nb, k, Xr, 1, nx_, 0, Tsh, nb, 1, 0, GD, nb, 1, 1);
          if (want_B) {
            double2* GXr = GX + (int64_t)r0 * S * nx_;
            if (tl) {
              dim3 g((unsigned)((k + 63) / 64), (unsigned)((cpt.maxklen + 79) / 80), (unsigned)cpt.tiles);
              (k_zgemm_gw_tiles<<<g, 256, 0, st>>>(ctt, Tsh, nb, k, cpt.krows, (double2*)B(P->o_bGWc), 0),
               ++g_launches);
              // written, not accumulated: gx_beta is set only for class (0,0),
              // one row, whose target is still zero here
              (k_gw_reduce<<<blocks(k * nx_), 256, 0, st>>>(ctt.tdesc, (const int32_t*)(ws + cpt.o_pos), cpt.tiles,
                                                           P->Kp[tcls], (const double2*)B(P->o_bGWc), cpt.krows, k,
                                                           GXr, nx_, nx_), ++g_launches);
            } else {
              zgemm(st, k, nx_, nb, Tsh, nb, 1, 0, D, 1, nb, 0, GXr, nx_, 1, gx_beta, bn);
            }
          }
        }
        if (tl)
          (k_gd_scatter<<<(unsigned)cpt.tiles, 256, 0, st>>>(ctt, (const double2*)B(P->o_bGDc), nb, GD), ++g_launches);
      };
      if (cls == 1)
        shifted(Lc[2], na, 0, ntp, (const double2*)(ws + P->o_X01), T.DTU, GT.DTU, (double2*)B(P->o_bGX01), 0, 64, 2);
      if (cls == 3)
        shifted(Lc[5], ntp, 1, na, (const double2*)(ws + P->o_X10), T.DT, GT.DT, (double2*)B(P->o_bGX10), 0, 16, -1);
      if (cls == 0)
        shifted(Lc[2], ntp, 1, ntp, (const double2*)(ws + P->o_X00), T.DTU, GT.DTU, (double2*)B(P->o_bGX00), 1, 64, 2);
      if (want_B && cls == 1 && Lc[2].n > 0)
        (k_gint<<<blocks((int64_t)nrow * na * ntp), 256, 0, st>>>(INT_X01, X.sp, (const double2*)B(P->o_bGX01), nrow,
                                                                 na * ntp, na * ntp, Gt, npair), ++g_launches);
      if (want_B && cls == 3 && Lc[5].n > 0)
        (k_gint<<<blocks((int64_t)nrow * ntp * na), 256, 0, st>>>(INT_X10, X.sp, (const double2*)B(P->o_bGX10), nrow,
                                                                 ntp * na, ntp * na, Gt, npair), ++g_launches);
    }
    // E0 term of the one-body coefficient, then the reference-state gradient
    (k_e0grad<<<blocks(na * na), 256, 0, st>>>(g1, scal, X.sp, Gf), ++g_launches);
    if (want_B && P->ntp > 0) {  // E0 term of <tu||vw>, then its pair-space coefficients
      const double2* g2 = (const double2*)(ws + P->o_g2 + P->g_stride * r);
      (k_x00e0<<<blocks((int64_t)P->ntp * P->ntp), 256, 0, st>>>(g1, g2, scal, P->ntp, (double2*)B(P->o_bGX00)),
       ++g_launches);
      (k_gint<<<blocks((int64_t)P->ntp * P->ntp), 256, 0, st>>>(INT_X00, X.sp, (const double2*)B(P->o_bGX00), P->ntp,
                                                                P->ntp, P->ntp, Gt, npair), ++g_launches);
    }
    if (g_c) {
      const struct { int fam, cls; double2* g; } sc[5] = {{FAM_T, 5, GT.DT}, {FAM_TD, 7, GT.DTD}, {FAM_TU, 2, GT.DTU},
                                                          {FAM_TDUD, 6, GT.DTDUD}, {FAM_TDU, 4, GT.DTDU}};
      for (const auto& q : sc)
        if (Lc[q.cls].n > 0)
          (k_dscatter<<<blocks(LP.n), 256, 0, st>>>(q.fam, Lc[q.cls], LP, P->das, X.binom, q.g, Gc), ++g_launches);
      (k_sigma<<<blocks(LP.n), 256, 0, st>>>(LP, Lc[4], Lc[2], P->das, X.sp, X.binom, T.DTDU, T.DTU,
                                             (const double2*)(ws + P->o_X00), X.f, sig), ++g_launches);
      (k_cbar<<<blocks(LP.n), 256, 0, st>>>(LP.n, Gc, c22, c, sig, scal, X.E0p + r, g1,
                                            (double2*)g_c + (int64_t)r * LP.n), ++g_launches);
    }
  }
  if (E2) launch_reduce(P, ws, st, E2, nullptr, nullptr);
  (k_nd<<<blocks(P->n), 256, 0, st>>>(X.sp, Nx, Nt, Nd), ++g_launches);
  if (g_h) (k_hbar<<<blocks((int64_t)P->n * P->n), 256, 0, st>>>(X.sp, Gf, Nd, (double2*)g_h), ++g_launches);
  if (want_B) {
    const int Lc_ = d.L_coulomb, Lx_ = d.L_extra, Lt = Lc_ + Lx_, n = P->n;
    double* GG = (double*)B(P->o_bGG);
    double2* Gh = (double2*)B(P->o_bGh);
    double2* Cs = (double2*)B(P->o_bCs);
    double2* GBc = (double2*)B(P->o_bGB);
    double2* ftr = (double2*)B(P->o_bFtr);
    double* gw = (double*)B(P->o_bGw);
    (k_gg<<<blocks((int64_t)n * n), 256, 0, st>>>(X.sp, Nd, Ntt, Ge, Gea, GG), ++g_launches);
    (k_symm<<<blocks(npair * npair), 256, 0, st>>>(Gt, npair, Gh), ++g_launches);
    zgemm(st, Lt, npair, npair, X.Bo, npair, 1, 0, Gh, 1, npair, 0, Cs, npair, 1, 0);
    (k_ftr<<<Lt, 256, 0, st>>>(X.sp, (const double2*)in->B_c, (const double2*)in->B_x, Lc_, Gf, ftr), ++g_launches);
    (k_bcoef<<<blocks((int64_t)Lt * n * n), 256, 0, st>>>(X.sp, (const double2*)in->B_c, (const double2*)in->B_x, Lc_,
                                                          Lx_, X.wt, X.dg, Cs, GG, Gf, ftr, GBc), ++g_launches);
    if (g_Bc || g_Bx)
      (k_bproj<<<blocks((int64_t)Lt * n * n), 256, 0, st>>>(n, Lc_, Lx_, GBc, (double2*)g_Bc, (double2*)g_Bx),
       ++g_launches);
    if (dE2_dlambda) {
      (k_gw<<<Lt, 256, 0, st>>>(X.sp, (const double2*)in->B_c, (const double2*)in->B_x, Lc_, X.Bo, Cs, GG, Gf, X.dg,
                                gw), ++g_launches);
      if (Lx_ > 0) (k_dlambda<<<1, 256, 0, st>>>(gw, in->w_x, Lc_, Lx_, dE2_dlambda), ++g_launches);
      else cudaMemsetAsync(dE2_dlambda, 0, sizeof(double), st);
    }
  }
  P->launches = g_launches;
  if (cudaGetLastError() != cudaSuccess) return E2_ERR_CUDA;
  return E2_OK;
}

e2_status e2_reference_workspace_size(const e2_problem* P, size_t* bytes) {
  if (!P || !bytes) return E2_ERR_INVALID_ARG;
  *bytes = P->solve_bytes;
  return E2_OK;
}

e2_status e2_reference_solve(e2_problem* P, const e2_inputs* in, double tol, int max_iter, void* workspace,
                             size_t workspace_bytes, void* stream_, double* c_out, double* E0_out, int* iters_out) {
  if (!P || !in || !c_out || !E0_out || !in->h || !in->B_c || !in->c) return E2_ERR_INVALID_ARG;
  if (P->d.L_extra > 0 && (!in->B_x || !in->w_x)) return E2_ERR_INVALID_ARG;
  if (!(tol > 0.0) || max_iter < 1) return E2_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < P->solve_bytes || ((uintptr_t)workspace & 255)) return E2_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream_;
  unsigned char* ws = (unsigned char*)workspace;
  cudaGetLastError();
  if (setup_common(P, in, ws, st) != E2_OK) return E2_ERR_CUDA;
  const int R = P->d.n_roots, mmax = P->sv_mmax;
  const DevList LP = dev_list(P, P->listP, ws);
  const int64_t np = LP.n;
  if (np < R) return E2_ERR_SHAPE;
  Ctx X = ctx(P, ws);
  Tabs T = tables(P, ws, 0);
  double2* V = (double2*)(ws + P->o_sV);
  double2* S = (double2*)(ws + P->o_sS);
  double2* Xv = (double2*)(ws + P->o_sX);
  double2* Rv = (double2*)(ws + P->o_sR);
  double2* Dv = (double2*)(ws + P->o_sD);
  double2* Tv = (double2*)(ws + P->o_sT);
  double2* Gd = (double2*)(ws + P->o_sG);
  double2* Yd = (double2*)(ws + P->o_sY);
  const DevList L11 = dev_list(P, P->list_of[4], ws), L02 = dev_list(P, P->list_of[2], ws);
  auto sigma = [&](const double2* v, double2* s) {
    build_tables(P, ws, st, v, T, false);
    (k_sigma<<<blocks(np), 256, 0, st>>>(LP, L11, L02, P->das, X.sp, X.binom, T.DTDU, T.DTU,
                                        (const double2*)(ws + P->o_X00), X.f, s), ++g_launches);
  };
  auto gram = [&](const double2* a, int na_, const double2* bb, int nb_) {
    std::vector<cd> out((size_t)na_ * nb_);
    (k_gram<<<na_ * nb_, 256, 0, st>>>(a, bb, np, nb_, Gd), ++g_launches);
    cudaMemcpyAsync(out.data(), Gd, 16 * out.size(), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return out;
  };
  auto upload = [&](const std::vector<cd>& y) {
    cudaMemcpyAsync(Yd, y.data(), 16 * y.size(), cudaMemcpyHostToDevice, st);
  };
  int k = 0;
  // copy a vector into slot k, orthogonalise it twice against slots < k, normalise, and build its sigma
  auto append = [&](const double2* src) -> bool {
    double2* vk = V + (int64_t)k * np;
    if (src != vk) cudaMemcpyAsync(vk, src, 16 * (size_t)np, cudaMemcpyDeviceToDevice, st);
    for (int pass = 0; pass < 2 && k > 0; ++pass) {
      std::vector<cd> ov = gram(V, k, vk, 1);
      for (auto& z : ov) z = -z;
      upload(ov);
      (k_lincomb<<<dim3(blocks(np), 1), 256, 0, st>>>(V, k, np, (const double2*)Yd, 1, 1, vk), ++g_launches);
    }
    double nrm = gram(vk, 1, vk, 1)[0].real();
    if (!(nrm > 1e-24)) return false;
    (k_scale<<<blocks(np), 256, 0, st>>>(vk, np, 1.0 / std::sqrt(nrm)), ++g_launches);
    sigma(vk, S + (int64_t)k * np);
    ++k;
    return true;
  };
  for (int j = 0; j < R; ++j)
    if (!append((const double2*)in->c + (int64_t)j * np)) return E2_ERR_SHAPE;
  std::vector<double> w;
  std::vector<cd> Y;
  int it = 0;
  for (; it < max_iter; ++it) {
    std::vector<cd> H = gram(V, k, S, k);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j <= i; ++j) {
        cd a = 0.5 * (H[(size_t)i * k + j] + std::conj(H[(size_t)j * k + i]));
        H[(size_t)i * k + j] = a;
        H[(size_t)j * k + i] = std::conj(a);
      }
    herm_eig(k, H, w, Y);
    std::vector<cd> Yr((size_t)k * R);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < R; ++j) Yr[(size_t)i * R + j] = Y[(size_t)i * k + j];
    upload(Yr);
    (k_lincomb<<<dim3(blocks(np), R), 256, 0, st>>>(V, k, np, (const double2*)Yd, R, 0, Xv), ++g_launches);
    (k_lincomb<<<dim3(blocks(np), R), 256, 0, st>>>(S, k, np, (const double2*)Yd, R, 0, Rv), ++g_launches);
    for (int j = 0; j < R; ++j)
      (k_residual<<<blocks(np), 256, 0, st>>>(Rv + (int64_t)j * np, Xv + (int64_t)j * np, LP.eA, np, w[j],
                                             Dv + (int64_t)j * np), ++g_launches);
    std::vector<cd> rn = gram(Rv, R, Rv, R);
    bool done = true;
    std::vector<int> open;
    for (int j = 0; j < R; ++j)
      if (std::sqrt(std::max(0.0, rn[(size_t)j * R + j].real())) >= tol) {
        done = false;
        open.push_back(j);
      }
    if (done) break;
    if (k + (int)open.size() > mmax) {  // restart from the Ritz vectors
      (k_lincomb<<<dim3(blocks(np), R), 256, 0, st>>>(S, k, np, (const double2*)Yd, R, 0, Tv), ++g_launches);
      cudaMemcpyAsync(V, Xv, 16 * (size_t)R * np, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(S, Tv, 16 * (size_t)R * np, cudaMemcpyDeviceToDevice, st);
      k = R;
    }
    int added = 0;
    for (int j : open)
      if (k < mmax && append(Dv + (int64_t)j * np)) ++added;
    if (added == 0) break;
  }
  cudaMemcpyAsync(c_out, Xv, 16 * (size_t)R * np, cudaMemcpyDeviceToDevice, st);
  double EOh = 0.0;
  cudaMemcpyAsync(&EOh, X.EO, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return E2_ERR_CUDA;
  for (int j = 0; j < R; ++j) E0_out[j] = w[j] + EOh;
  if (iters_out) *iters_out = it;
  return E2_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ fixed scratch variant

// Scratch for e2_forward_noalloc, compiled into the library: every device
// that loads it holds these bytes until the process exits.  Nothing in the
// forward layout needs to start at zero (every buffer is fully written before
// it is read), so calls do not clear it; consecutive calls simply overwrite it.
static __device__ __align__(256) unsigned char e2_static_scratch[E2_STATIC_SCRATCH_BYTES];

namespace {
std::mutex g_scratch_mu;
void* g_scratch_ptr[128] = {};  // device address of e2_static_scratch, per device ordinal
}  // namespace

extern "C" e2_status e2_forward_noalloc(e2_problem* P, const e2_inputs* in, void* stream, double* E2,
                                        double* E2_class, double* E0) {
  if (!P) return E2_ERR_INVALID_ARG;
  if (P->ws_bytes > (size_t)E2_STATIC_SCRATCH_BYTES) return E2_ERR_WORKSPACE;  // before any GPU call
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return E2_ERR_CUDA;
  void* ptr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      // once per device, with that device current: the host-side symbol is only
      // a stand-in, the kernels need the array's device address
      if (cudaGetSymbolAddress(&g_scratch_ptr[dev], e2_static_scratch) != cudaSuccess) {
        g_scratch_ptr[dev] = nullptr;
        return E2_ERR_CUDA;
      }
    }
    ptr = g_scratch_ptr[dev];
  }
  return e2_forward(P, in, ptr, (size_t)E2_STATIC_SCRATCH_BYTES, stream, E2, E2_class, E0);
}
