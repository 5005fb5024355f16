// Host plan: occupation patterns, string lists, column tiles and the
// workspace layout of a problem; the C entry points that create and query it.
#include "e2_host.h"

#include <cstring>
#include <new>
#include <queue>

namespace e2 {

int64_t binom_h(int n, int k) {
  if (k < 0 || n < 0 || k > n) return 0;
  int64_t r = 1;
  int kk = std::min(k, n - k);
  for (int j = 1; j <= kk; ++j) r = r * (n - kk + j) / j;
  return r;
}

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
  }
  // width of the backward's compacted product tiles: every padded row is a
  // full row of FP64 tensor work, so take the width that pads the tiles'
  // lengths least (the widest of those within 1% of the least)
  {
    int64_t best = -1;
    for (int bn : {80, 64, 48, 32}) {
      int64_t padded = 0;
      for (int64_t j = 0; j < cp.tiles; ++j) padded += (cp.tdesc[4 * j + 1] + bn - 1) / bn * bn;
      if (best < 0 || padded * 100 < best * 99) {
        best = padded;
        cp.pbn = bn;
      }
    }
    cp.gd_ctas = 0;
    for (int64_t j = 0; j < cp.tiles; ++j) cp.gd_ctas += (cp.tdesc[4 * j + 1] + cp.pbn - 1) / cp.pbn;
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
    P->q_full[c] = P->q_per_class[c];
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
  P->o_xc = ws.take(sizeof(int32_t) * std::max(1, P->ncc));
  P->o_xv = ws.take(sizeof(int32_t) * std::max(1, P->nvc));
  P->xc.assign(std::max(1, P->ncc), -1);
  P->xv.assign(std::max(1, P->nvc), -1);
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
  P->o_status = ws.take(sizeof(unsigned long long) * (1 + (size_t)R * E2_NCLASS));
  P->o_EO = ws.take(sizeof(double));
  P->o_E0p = ws.take(sizeof(double) * R);
  P->o_E0 = ws.take(sizeof(double) * R);
  P->o_G = ws.take(sizeof(double) * P->n * P->n);
  P->o_epsh = ws.take(sizeof(double) * P->n);
  P->o_dg = ws.take(sizeof(double) * Lt * P->n);
  P->o_wt = ws.take(sizeof(double) * Lt);
  P->o_Bo = ws.take(16 * (size_t)Lt * P->n * P->nocc);
  P->o_f = ws.take(16 * (size_t)P->n * P->nocc);
  // Sliced bf16 contraction: classes whose real contraction length 2 Kp is at
  // most 256 (the exactness bound of the level sums), when the slices and the
  // float-float tables take at most 16 GiB in all.
  {
    size_t extra = 0;
    std::vector<bool> ldf(P->lists.size(), false);
    for (int c : {2, 5, 7, 6}) {
      const int li = P->list_of[c];
      P->oz_ok[c] = ((d.class_mask >> c) & 1u) && P->M[c] > 0 && li >= 0 && P->lists[li].n > 0 && 2 * P->Kp[c] <= 256;
      if (!P->oz_ok[c]) continue;
      P->oz_kq[c] = (2 * P->Kp[c] + 31) / 32 * 32;
      P->oz_mpad[c] = (P->M[c] + 63) / 64 * 64;
      P->oz_npad[c] = (P->lists[li].n + 63) / 64 * 64;
      extra += (size_t)2 * OZ_S * P->oz_kq[c] * (P->oz_mpad[c] + 2 * P->oz_npad[c]);
      if (!ldf[li]) extra += 8 * (size_t)(P->nx + 2) * P->lists[li].n;
      ldf[li] = true;
    }
    // the class-(2,2) list's tables too (its float-float adjoint)
    const int l8 = P->list_of[8];
    const bool d8 = ((d.class_mask >> 8) & 1u) && P->M[8] > 0 && l8 >= 0 && P->lists[l8].n > 0;
    if (d8 && !ldf[l8]) extra += 8 * (size_t)(P->nx + 2) * P->lists[l8].n;
    const bool fits = extra <= (size_t(16) << 30);
    for (int c : {2, 5, 7, 6}) {
      P->oz_ok[c] = P->oz_ok[c] && fits;
      P->use_oz[c] = false;  // FP64 by default; the sliced form is opt-in
      if (P->oz_ok[c]) P->lists[P->list_of[c]].df = true;
    }
    if (d8 && fits) P->lists[l8].df = true;
    P->oz_ok[8] = d8 && fits;  // class (2,2) in float-float (opt-in)
    P->use_oz[8] = false;
  }
  for (HostList& L : P->lists) {
    L.o_str = ws.take(sizeof(uint64_t) * std::max<int64_t>(L.n, 1));
    L.o_eA = ws.take(sizeof(double) * std::max<int64_t>(L.n, 1));
    L.o_U = ws.take(sizeof(double) * (size_t)(P->nx + 1) * std::max<int64_t>(L.n, 1));
    if (L.df) {
      L.o_eAdf = ws.take(8 * (size_t)L.n);
      L.o_Udf = ws.take(8 * (size_t)(P->nx + 1) * L.n);
    }
  }
  const int dense[5] = {2, 5, 7, 4, 6};
  for (int c = 0; c < E2_NCLASS; ++c) P->o_rows[c] = P->o_W[c] = 0;
  for (int c : dense) {
    if (P->M[c] == 0) continue;
    P->o_rows[c] = ws.take(sizeof(RowInfo) * P->M[c]);
    P->o_W[c] = ws.take(16 * (size_t)P->M[c] * P->Kp[c]);
    if (P->oz_ok[c]) {
      P->o_ozA[c] = ws.take((size_t)2 * OZ_S * P->oz_mpad[c] * P->oz_kq[c]);
      P->o_ozRx[c] = ws.take(4 * (size_t)P->oz_mpad[c]);
    }
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
  for (int c : {2, 5, 7, 6})
    if (P->oz_ok[c]) {
      P->o_ozB[c] = ws.take((size_t)2 * OZ_S * 2 * P->oz_npad[c] * P->oz_kq[c]);
      P->o_ozCx[c] = ws.take(4 * (size_t)P->oz_npad[c]);
    }
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
    // slices of the factor-index products on the sliced GEMM: the largest of
    // (ai|bt), (at|bu) (B sliced over all n_v n_a columns) and (av|uw)
    if (Lt > 0 && nva > 0) {
      size_t b = zgemm_sliced_bytes(nva, nva, Lt);
      b = std::max(b, zgemm_sliced_bytes((int64_t)P->nvc * P->ncc, nva, Lt));
      b = std::max(b, zgemm_sliced_bytes(nva, (int64_t)P->na * P->na, Lt));
      P->o_ozS = P->o_vaX + al(P->va_cap);
      P->ozS_bytes = b;
      P->use_oz_setup = false;
      ws.top = std::max(ws.top, P->o_ozS + al(b));
    }
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
      const int64_t Nt = (Nc + 63) / 64 * 64;  // amplitude rows in tile order are 64 x tiles wide
      int64_t rows_fit = (int64_t)(tbudget / (16 * (size_t)Nt)) / 64 * 64;
      if (P->cplan[c].built)  // compacted Gamma_W of a chunk: rows x compacted columns
        rows_fit = std::min<int64_t>(rows_fit, (int64_t)(gwbudget / (16 * (size_t)P->cplan[c].krows)) / 64 * 64);
      rows_fit = std::max<int64_t>(64, rows_fit);
      P->chunk_rows[c] = std::min<int64_t>(rows_fit, (Mc + 63) / 64 * 64);
      const int64_t ct = (Nc + 63) / 64;
      tmax = std::max(tmax, (size_t)16 * P->chunk_rows[c] * Nt);
      if (P->cplan[c].built) {
        gdc = std::max(gdc, (size_t)16 * P->cplan[c].krows * 64);
        gwc = std::max(gwc, (size_t)16 * P->chunk_rows[c] * P->cplan[c].krows);
      }
      // per-tile sums of one row chunk, reduced before the next chunk
      const int64_t rtc = P->chunk_rows[c] / 64;
      hrow = std::max(hrow, (size_t)8 * P->chunk_rows[c] * ct);
      hcol = std::max(hcol, (size_t)8 * rtc * Nc);
      scalt = std::max(scalt, (size_t)16 * rtc * ct);
      hsum = std::max(hsum, (size_t)8 * Mc);
    }
    for (size_t li = 0; li < P->lists.size(); ++li) hA = std::max(hA, (size_t)8 * P->lists[li].n);
    size_t gmax = 8;
    for (int c : {1, 3, 0})
      if (P->list_of[c] >= 0) gmax = std::max(gmax, (size_t)P->M[c] * P->lists[P->list_of[c]].n);
    const int64_t nyb = (int64_t)P->nvb * (P->nvb + 1) / 2;
    const int64_t np22 = lsize(8), xb22 = (np22 + 255) / 256;
    // class (2,2) adjoint in chunks of core pairs whose partials fit 2 GiB
    const size_t per_z = 8 * (size_t)nyb * (2 * (size_t)std::max<int64_t>(np22, 1) + 19 * (size_t)std::max<int64_t>(xb22, 1));
    P->z22_chunk = (int)std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(P->ncp, 1),
                                                             (int64_t)((size_t(2) << 30) / std::max<size_t>(per_z, 1))));
    const size_t yz = (size_t)std::max<int64_t>(1, nyb * P->z22_chunk);
    P->z22_plan = P->z22_chunk;
    for (int c = 0; c < E2_NCLASS; ++c) P->chunk_rows_plan[c] = P->chunk_rows[c];
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
    size_t hm = 8, hocc = 8, tsh = 16;
    for (int c = 0; c < E2_NCLASS; ++c) P->o_bGW[c] = 0;
    for (int c : {2, 5, 7, 4, 6}) {
      const int64_t Mc = P->M[c], Nc = lsize(c);
      if (Mc == 0 || Nc == 0) continue;
      P->o_bGW[c] = ws.take(16 * (size_t)Mc * P->Kp[c]);
      hm = std::max(hm, (size_t)8 * P->chunk_rows[c] * ((Nc + 63) / 64 * 64));
      hocc = std::max(hocc, (size_t)8 * Mc * P->na);
    }
    const int64_t M22 = P->ncp * P->nvp;
    hocc = std::max(hocc, (size_t)8 * std::max<int64_t>(M22, 1) * P->na);
    for (int c : {1, 3, 0})
      if (P->list_of[c] >= 0) hocc = std::max(hocc, (size_t)8 * P->M[c] * P->na);
    // marginals of the per-row sums over hole / particle tuples (at most
    // C(n_vc,2) particle and C(n_cc,2) hole tuples)
    const size_t tp = (size_t)std::max<int64_t>(std::max<int64_t>(pairs(P->nvc), P->nvc), 1);
    const size_t th = (size_t)std::max<int64_t>(std::max<int64_t>(pairs(P->ncc), P->ncc), 1);
    const size_t zz = 8 * (tp * (1 + (size_t)P->na) + th * (1 + (size_t)P->na + (size_t)std::max(P->nvc, 1)));
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
    // slices of the adjoint's products on the sliced GEMM: Gamma_D and
    // Gamma_W of a row chunk of each dense class, and Cs = B Gamma^ when its
    // slices take at most 4 GiB (else Cs stays on the FP64 pipe)
    {
      size_t oz = 0;
      for (int c : {2, 5, 7, 4, 6}) {
        const int64_t Nc = lsize(c), Mc = P->chunk_rows[c];
        if (P->M[c] == 0 || Nc == 0 || Mc == 0) continue;
        oz = std::max(oz, zgemm_sliced_bytes(Nc, P->Kp[c], Mc, OZ_ADJ_S));
        oz = std::max(oz, zgemm_sliced_bytes(Mc, P->Kp[c], Nc, OZ_ADJ_S));
      }
      // shifted amplitudes of the gather classes: (table list, shifts S, width nx, rows)
      struct Sh { int lcls; int64_t S, nx, rows; };
      const Sh shs[3] = {{2, P->na, P->ntp, P->nvc}, {5, P->ntp, P->na, P->ncc}, {2, P->ntp, P->ntp, 1}};
      const int gcls[3] = {1, 3, 0};
      for (int q = 0; q < 3; ++q) {
        const int64_t nb = lsize(shs[q].lcls);
        if (P->list_of[gcls[q]] < 0 || nb == 0 || shs[q].S == 0 || shs[q].nx == 0) continue;
        const int64_t k = std::max<int64_t>(
            1, std::min<int64_t>(shs[q].rows * shs[q].S, (int64_t)(P->tsh_bytes / (16 * (size_t)nb))) / shs[q].S *
                   shs[q].S);
        oz = std::max(oz, zgemm_sliced_bytes(nb, shs[q].nx, k, OZ_ADJ_S));
        oz = std::max(oz, zgemm_sliced_bytes(k, shs[q].nx, nb, OZ_ADJ_S));
      }
      const size_t cs = Lt > 0 ? zgemm_sliced_bytes(Lt, npair, npair, OZ_ADJ_S) : 0;
      if (cs <= (size_t(4) << 30)) oz = std::max(oz, cs);
      P->bOz_bytes = oz;
      P->use_oz_adj = false;
      P->o_bOz = ws.take(std::max<size_t>(oz, 256));
      P->o_bC2 = ws.take(8 * (size_t)std::max<int64_t>(lsize(8), 1));
    }
    P->bwd_bytes = ws.top;
  }

  // ---- host image of the plan region
  P->plan_blob.assign(P->plan_bytes, 0);
  auto rel = [&](size_t o) { return o - P->o_plan; };
  put(P->plan_blob, rel(P->o_cc), P->cc.data(), P->cc.size());
  put(P->plan_blob, rel(P->o_vc), P->vc.data(), P->vc.size());
  put(P->plan_blob, rel(P->o_xc), P->xc.data(), P->xc.size());
  put(P->plan_blob, rel(P->o_xv), P->xv.data(), P->xv.size());
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

}  // namespace e2

using namespace e2;

extern "C" {

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
  if (!P) return E2_ERR_OOM;
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
  } catch (const std::bad_alloc&) {
    st = E2_ERR_OOM;
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

e2_status e2_set_external_das(e2_problem* P, int n_cdas, const int32_t* core_size, const int32_t* core_max_holes,
                              int n_vdas, const int32_t* virt_size, const int32_t* virt_max_particles) {
  if (!P || n_cdas < 0 || n_vdas < 0 || n_cdas > 64 || n_vdas > 64) return E2_ERR_INVALID_ARG;
  if ((n_cdas && (!core_size || !core_max_holes)) || (n_vdas && (!virt_size || !virt_max_particles)))
    return E2_ERR_INVALID_ARG;
  // subspace of every core / virtual spinor (consecutive blocks in global order)
  std::vector<int32_t> csub(P->d.n_core, -1), vsub(P->d.n_virt, -1);
  int64_t at = 0;
  for (int s = 0; s < n_cdas; ++s) {
    if (core_size[s] < 1 || core_max_holes[s] < 1 || at + core_size[s] > P->d.n_core) return E2_ERR_INVALID_ARG;
    for (int k = 0; k < core_size[s]; ++k) csub[at++] = core_max_holes[s] == 1 ? s : -1;
  }
  if (n_cdas && at != P->d.n_core) return E2_ERR_INVALID_ARG;
  at = 0;
  for (int s = 0; s < n_vdas; ++s) {
    if (virt_size[s] < 1 || virt_max_particles[s] < 1 || at + virt_size[s] > P->d.n_virt) return E2_ERR_INVALID_ARG;
    for (int k = 0; k < virt_size[s]; ++k) vsub[at++] = virt_max_particles[s] == 1 ? s : -1;
  }
  if (n_vdas && at != P->d.n_virt) return E2_ERR_INVALID_ARG;
  bool any = false;
  for (int i = 0; i < P->ncc; ++i) {
    P->xc[i] = csub[P->cc[i]];
    any = any || P->xc[i] >= 0;
  }
  for (int a = 0; a < P->nvc; ++a) {
    P->xv[a] = vsub[P->vc[a] - P->nocc];
    any = any || P->xv[a] >= 0;
  }
  P->ext_das = any;
  auto rel = [&](size_t o) { return o - P->o_plan; };
  std::memcpy(P->plan_blob.data() + rel(P->o_xc), P->xc.data(), sizeof(int32_t) * P->xc.size());
  std::memcpy(P->plan_blob.data() + rel(P->o_xv), P->xv.data(), sizeof(int32_t) * P->xv.size());
  // class sizes: allowed hole pairs times allowed particle pairs times strings
  int64_t hp = 0, pp = 0;  // pairs of one limited subspace
  for (int i = 0; i < P->ncc; ++i)
    for (int j = i + 1; j < P->ncc; ++j) hp += P->xc[i] >= 0 && P->xc[i] == P->xc[j];
  for (int a = 0; a < P->nvc; ++a)
    for (int b = a + 1; b < P->nvc; ++b) pp += P->xv[a] >= 0 && P->xv[a] == P->xv[b];
  const double hc = (double)(P->ncp - hp) / std::max<double>((double)P->ncp, 1.0);
  const double vc = (double)(P->nvp - pp) / std::max<double>((double)P->nvp, 1.0);
  const double frac[E2_NCLASS] = {1, 1, vc, 1, 1, vc, hc, hc, hc * vc};
  for (int c = 0; c < E2_NCLASS; ++c) P->q_per_class[c] = P->q_full[c] * frac[c];
  for (int c : {2, 5, 6, 7, 8})  // exact integers
    if (P->list_of[c] >= 0)
      P->q_per_class[c] = (double)(c == 2 ? P->nvp - pp : c == 5 ? (int64_t)P->ncc * (P->nvp - pp)
                                   : c == 6 ? P->ncp - hp : c == 7 ? (P->ncp - hp) * (int64_t)P->nvc
                                                          : (P->ncp - hp) * (P->nvp - pp)) *
                          (double)P->lists[P->list_of[c]].n;
  return E2_OK;
}

e2_status e2_set_contraction(e2_problem* P, int cls, int mode) {
  if (!P || cls < E2_CONTRACT_ADJOINT || cls >= E2_NCLASS || (mode != E2_CONTRACT_FP64 && mode != E2_CONTRACT_SLICED))
    return E2_ERR_INVALID_ARG;
  if (cls == E2_CONTRACT_ADJOINT) {
    if (mode == E2_CONTRACT_SLICED && P->bOz_bytes == 0) return E2_ERR_UNSUPPORTED;
    P->use_oz_adj = mode == E2_CONTRACT_SLICED;
    return E2_OK;
  }
  if (cls == E2_CONTRACT_SETUP) {
    if (mode == E2_CONTRACT_SLICED && P->ozS_bytes == 0) return E2_ERR_UNSUPPORTED;
    P->use_oz_setup = mode == E2_CONTRACT_SLICED;
    return E2_OK;
  }
  if (mode == E2_CONTRACT_SLICED && !P->oz_ok[cls]) return E2_ERR_UNSUPPORTED;
  P->use_oz[cls] = mode == E2_CONTRACT_SLICED;
  return E2_OK;
}

e2_status e2_contraction(const e2_problem* P, int cls, int* mode, int* sliced_available) {
  if (!P || cls < E2_CONTRACT_ADJOINT || cls >= E2_NCLASS) return E2_ERR_INVALID_ARG;
  const bool on = cls == E2_CONTRACT_ADJOINT ? P->use_oz_adj
                  : cls == E2_CONTRACT_SETUP ? P->use_oz_setup
                                             : P->use_oz[cls];
  const bool ok = cls == E2_CONTRACT_ADJOINT ? P->bOz_bytes > 0
                  : cls == E2_CONTRACT_SETUP ? P->ozS_bytes > 0
                                             : P->oz_ok[cls];
  if (mode) *mode = on ? E2_CONTRACT_SLICED : E2_CONTRACT_FP64;
  if (sliced_available) *sliced_available = ok ? 1 : 0;
  return E2_OK;
}

e2_status e2_set_adjoint_chunks(e2_problem* P, int64_t rows, int core_pairs) {
  if (!P) return E2_ERR_INVALID_ARG;
  for (int c = 0; c < E2_NCLASS; ++c) {
    const int64_t plan = P->chunk_rows_plan[c];
    P->chunk_rows[c] = (rows <= 0 || plan == 0) ? plan : std::min<int64_t>(plan, std::max<int64_t>(64, rows / 64 * 64));
  }
  P->z22_chunk = core_pairs <= 0 ? P->z22_plan : std::min(P->z22_plan, core_pairs);
  return E2_OK;
}

e2_status e2_set_class_tiles(e2_problem* P, int cls, int on) {
  if (!P || cls < 0 || cls >= E2_NCLASS) return E2_ERR_INVALID_ARG;
  if (on && !P->cplan[cls].built) return E2_ERR_UNSUPPORTED;
  P->use_cols[cls] = on != 0;
  return E2_OK;
}

}  // extern "C"
