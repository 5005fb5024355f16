// C ABI: the stream-ordered launch helpers and e2_forward (with its
// allocation-free variant), the sampled-partials hook, the autotuner and the
// measurement hooks.  No device allocation.
#include "e2_host.h"

#include <cstdio>
#include <cstring>
#include <string>

namespace e2 {

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

// kernels enqueued by the current host thread (read back as the count of one call)
thread_local int64_t g_launches = 0;

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
  sp.xc = (const int32_t*)(ws + P->o_xc);
  sp.xv = (const int32_t*)(ws + P->o_xv);
  return X;
}

// Base of root r's D-table slot (offsets o_DT... apply to it): slot 0 inside
// the layout, or for a batch slot r >= 1 after the job's forward layout.
unsigned char* slot_base(const e2_problem* P, unsigned char* ws, int r) {
  if (!P->multi_slot) return ws;
  const int s = P->slots > 0 ? r % P->slots : r;
  if (s == 0) return ws;
  return ws + P->ws_bytes + (size_t)(s - 1) * P->d_stride - P->o_dstart;
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

OzOperands oz_operands(const e2_problem* P, unsigned char* ws, int r, int cls) {
  const HostList& L = P->lists[P->list_of[cls]];
  unsigned char* sb = slot_base(P, ws, r);
  return OzOperands{(const __nv_bfloat16*)(ws + P->o_ozA[cls]), P->oz_mpad[cls], (const int*)(ws + P->o_ozRx[cls]),
                    (const __nv_bfloat16*)(sb + P->o_ozB[cls]), P->oz_npad[cls], (const int*)(sb + P->o_ozCx[cls]),
                    P->oz_kq[cls], (const float2*)(ws + L.o_Udf), (const float2*)(ws + L.o_eAdf), P->nx};
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
// at C[m*csm + n*csn].  Tile width bn = 64, 16 or 24.  With `part` given and few
// output tiles, K is split into segments summed in a fixed order (the output
// region C[0 .. M*N) must then be dense in C's layout).
void zgemm(cudaStream_t st, int64_t M, int64_t N, int64_t K, const double2* A, int64_t sam, int64_t sak, int conjA,
           const double2* B, int64_t sbk, int64_t sbn, int conjB, double2* C, int64_t csm, int64_t csn, int beta,
           int bn) {
  if (M <= 0 || N <= 0) return;
  if (bn == 16 && N % 24 == 0 && N % 16 != 0) bn = 24;  // 24 active spinors: no padded columns
  const int bm = bn == 64 ? 64 : 128;  // tiles 64 x 64, 128 x 16 or 128 x 24
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
  else if (bn == 24)
    (k_zgemm24<<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, conjA, B, sbk, sbn, conjB, out, om, on, b, kseg, czs, -1),
     ++g_launches);
  else
    (k_zgemm64<<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, conjA, B, sbk, sbn, conjB, out, om, on, b, kseg, czs, -1),
     ++g_launches);
  if (nseg > 1) (k_zacc<<<blocks(M * N), 256, 0, st>>>(out, nseg, czs, M, N, C, csm, csn, beta), ++g_launches);
}

// Everything that depends only on the Hamiltonian and the partition:
// binomials, compact factors, G, eps^, f, E_O, string lists with e_A and U,
// and the active two-electron block <tu||vw>.
e2_status setup_common(e2_problem* P, const e2_inputs* in, unsigned char* ws, cudaStream_t st, bool upload) {
  const e2_desc& d = P->d;
  const int n = P->n, nocc = P->nocc, Lt = d.L_coulomb + d.L_extra;
  Ctx X = ctx(P, ws);
  // status word: no flags, every smallest |D| at the largest key
  (k_status_init<<<1, 256, 0, st>>>(status_word(P, ws), 1 + d.n_roots * E2_NCLASS), ++g_launches);
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
    const HostList& H = P->lists[li];
    // float-float copies of e_A and U, read only by the sliced kernels
    bool df_used = P->use_oz_adj && (int)li == P->list_of[8];
    for (int c : {2, 5, 7, 6, 8}) df_used = df_used || (P->use_oz[c] && P->list_of[c] == (int)li);
    if (H.df && df_used)
      (k_oz_tables<<<blocks((int64_t)(P->nx + 1) * L.n), 256, 0, st>>>(L.eA, L.U, L.n, P->nx + 1,
                                                                      (float2*)(ws + H.o_eAdf),
                                                                      (float2*)(ws + H.o_Udf)), ++g_launches);
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
      if (!(P->use_oz_setup && zgemm_sliced(st, (int64_t)P->nvc * P->ncc, nva, Lt, (const double2*)(ws + P->o_xYc), Lt,
                                            1, 0, Zf, nva, 1, 0, X12, nva, 1, 0, -1, ws + P->o_ozS, P->ozS_bytes)))
        zgemm(st, (int64_t)P->nvc * P->ncc, nva, Lt, (const double2*)(ws + P->o_xYc), Lt, 1, 0, Zf, nva, 1, 0, X12, nva,
              1, 0);
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
        // sliced: the factor columns of all n_v n_a pairs are cut once and
        // kept for the following stripes
        if (!(P->use_oz_setup && zgemm_sliced(st, rows, ldx, Lt, Yw + r0 * Lt, Lt, 1, 0, Zf, nva, 1, 0, Xv, ldx, 1, 0,
                                              r0, ws + P->o_ozS, P->ozS_bytes, nva, b0 > 0)))
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
    if (!(P->use_oz_setup && zgemm_sliced(st, nva, (int64_t)na * na, Lt, Yw, Lt, 1, 0, (const double2*)(ws + P->o_xZaa),
                                          (int64_t)na * na, 1, 0, X01g, (int64_t)na * na, 1, 0, -1, ws + P->o_ozS,
                                          P->ozS_bytes)))
      zgemm(st, nva, (int64_t)na * na, Lt, Yw, Lt, 1, 0, (const double2*)(ws + P->o_xZaa), (int64_t)na * na, 1, 0,
            X01g, (int64_t)na * na, 1, 0);
    (k_x01<<<blocks((int64_t)P->nvc * na * P->ntp), 256, 0, st>>>(X.sp, X01g, (double2*)(ws + P->o_X01)), ++g_launches);
  }
  if (P->part_cnt[3] > 0)
    (k_integrals<<<blocks((int64_t)P->ncc * P->ntp * na), 256, 0, st>>>(INT_X10, X.sp, X.Bo, X.wt, Lt, X.f, P->ncc,
                                                                       P->ntp * na, P->ntp * na, ws + P->o_X10), ++g_launches);
  // external subspace limits: the excluded rows' W rows and |<ab||ij>|^2 to zero
  if (P->ext_das) {
    for (int c : {2, 5, 7, 6})
      if (P->M[c] > 0 && P->part_cnt[c] > 0)
        (k_mask_rows<<<blocks(P->M[c] * P->Kp[c]), 256, 0, st>>>((double2*)(ws + P->o_W[c]), P->M[c], P->Kp[c],
                                                                (const RowInfo*)(ws + P->o_rows[c])), ++g_launches);
    if (P->part_cnt[8] > 0)
      (k_mask22<<<blocks(P->ncp * P->nvp), 256, 0, st>>>(ws + P->o_G22, P->ncp, P->nvp, X.sp, 0), ++g_launches);
  }
  // row slices of W for the classes on the sliced contraction
  for (int c : {2, 5, 7, 6})
    if (P->use_oz[c] && P->part_cnt[c] > 0)
      launch_slice_rows(st, (const double2*)(ws + P->o_W[c]), P->Kp[c], 1, P->M[c], P->Kp[c], P->oz_kq[c],
                        P->oz_mpad[c], (__nv_bfloat16*)(ws + P->o_ozA[c]), (int*)(ws + P->o_ozRx[c]));
}


// Gamma_D of a column-tiled class in compacted form, GDc (+)= per tile
// W[:, klist]^T conj(T[:, perm]) over the chunk's Mc rows, split-K as zgemm.
void zgemm_gd_tiles(cudaStream_t st, const ColPlan& cp, const ColTiles& ctl, const double2* W, int Kp,
                    const double2* T, int64_t N, int64_t Mc, double2* GDc, int beta, int conjT, int64_t t_ld) {
  const int64_t czs = cp.krows * 64;
  const int nseg = splitk_segments(cp.gd_ctas, Mc, 16 * (size_t)czs);
  const int64_t kseg = (Mc + nseg - 1) / nseg;
  dim3 grid((unsigned)((cp.maxklen + cp.pbn - 1) / cp.pbn), (unsigned)cp.tiles, (unsigned)nseg);
  if (nseg == 1) {
    launch_gd_tiles(cp.pbn, grid, st, ctl, W, Kp, T, N, Mc, GDc, beta, kseg, 0, conjT, t_ld);
    return;
  }
  double2* part = (double2*)g_splitk;
  launch_gd_tiles(cp.pbn, grid, st, ctl, W, Kp, T, N, Mc, part, 0, kseg, czs, conjT, t_ld);
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
  for (int cls : {2, 5, 7, 6})
    if (P->use_oz[cls] && P->part_cnt[cls] > 0) {
      const int64_t N = P->lists[P->list_of[cls]].n;
      unsigned char* sb = slot_base(P, ws, r);
      launch_slice_cols(st, Dcls[cls], N, 1, P->Kp[cls], N, P->oz_kq[cls], P->oz_npad[cls],
                        (__nv_bfloat16*)(sb + P->o_ozB[cls]), (int*)(sb + P->o_ozCx[cls]));
    }
  double2* g1 = (double2*)(ws + P->o_g1 + P->g_stride * r);
  double2* g2 = (double2*)(ws + P->o_g2 + P->g_stride * r);
  (k_gram<<<1 + na * na, 256, 0, st>>>(T.DTDU, T.DTDU, L11.n, 1 + na * na, g1), ++g_launches);
  if (P->ntp > 0 && L02.n > 0) (k_gram<<<P->ntp * P->ntp, 256, 0, st>>>(T.DTU, T.DTU, L02.n, P->ntp, g2), ++g_launches);
  else cudaMemsetAsync(g2, 0, 16 * (size_t)std::max(P->ntp * P->ntp, 1), st);
  (k_e0<<<1, 256, 0, st>>>(g1, g2, X.f, (const double2*)(ws + P->o_X00), X.sp, P->ntp, X.EO, X.E0p + r, X.E0d + r),
   ++g_launches);
}

// E2_class and E2 of every root from the partial slots (fixed order).
void launch_reduce(e2_problem* P, unsigned char* ws, cudaStream_t st, double* E2, double* E2_class, double* E0) {
  const int R = P->d.n_roots;
  double* e2c = E2_class ? E2_class : (double*)(ws + P->o_e2c);
  (k_reduce<<<R * E2_NCLASS, 256, 0, st>>>((const double*)(ws + P->o_part), (const int64_t*)(ws + P->o_partoff),
                                           (const int64_t*)(ws + P->o_partcnt), (const double2*)(ws + P->o_g1),
                                           (int)(P->g_stride / 16), R, e2c), ++g_launches);
  (k_finalize<<<1, 32, 0, st>>>(e2c, R, E2, (const double*)(ws + P->o_E0), E0, status_word(P, ws),
                                P->d.level_shift_b), ++g_launches);
}

}  // namespace e2

using namespace e2;

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
    case E2_ERR_INTRUDER: return "intruder state: |E0 - H_KK| below 1e-12 Eh without a level shift";
    case E2_ERR_OOM: return "out of host memory";
    case E2_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
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
  // with shards every rank writes only its own slots: the others stay 0, so
  // that a sum of the ranks' partials over ranks is exactly the unsharded set
  if (P->shard_n > 1) cudaMemsetAsync(part, 0, sizeof(double) * (size_t)part_total(P), st);
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
      int64_t u0, u1;  // row tiles of this rank (all of them without shards)
      shard_range(P, cls, u0, u1);
      if (u1 <= u0) continue;
      const DevList& L = Lc[cls];
      dim3 grid((unsigned)(u1 - u0), (unsigned)((L.n + 63) / 64));
      mark(cls, 0);
      if (P->use_oz[cls])
        launch_class_oz(st, cls, oz_operands(P, ws, r, cls), P->M[cls], L.n, (const RowInfo*)(ws + P->o_rows[cls]),
                        X.E0p + r, b, poff(cls), dmin_slot(P, ws, r, cls), u0, u1 - u0);
      else
        (k_class_gemm<<<grid, 256, 0, st>>>((const double2*)(ws + P->o_W[cls]), Dfor[cls], P->M[cls], L.n, P->Kp[cls],
                                           (const RowInfo*)(ws + P->o_rows[cls]), L.U, L.eA, X.E0p + r, b, poff(cls),
                                           AdjOut{}, col_tiles(P, ws, r, cls), dmin_slot(P, ws, r, cls),
                                           (P->M[cls] + 63) / 64, u0),
         ++g_launches);
      mark(cls, 1);
    }
    launch_sparse_classes(P, ws, st, r, c, mark);
  }
  double* e2c = E2_class ? E2_class : (double*)(ws + P->o_e2c);
  (k_reduce<<<R * E2_NCLASS, 256, 0, st>>>(part, (const int64_t*)(ws + P->o_partoff), (const int64_t*)(ws + P->o_partcnt),
                                          (const double2*)(ws + P->o_g1), (int)(P->g_stride / 16), R, e2c), ++g_launches);
  (k_finalize<<<1, 32, 0, st>>>(e2c, R, E2, X.E0d, E0, status_word(P, ws), b), ++g_launches);
  P->launches = g_launches;
  if (cudaGetLastError() != cudaSuccess) return E2_ERR_CUDA;
  return E2_OK;
}

e2_status e2_coupling_tables(e2_problem* P, const e2_inputs* in, void* workspace, size_t workspace_bytes,
                             void* stream_, int root, int family, double* table, uint64_t* strings, int64_t* rows,
                             int64_t* n_A) {
  if (!P || family < 0 || family > 4 || root < 0 || root >= P->d.n_roots) return E2_ERR_INVALID_ARG;
  const int na = P->na;
  const int cls_of[5] = {5, 7, 2, 6, 4};  // the class whose list each family's strings form
  const int64_t nrow = family <= 1 ? na : family <= 3 ? (int64_t)na * (na - 1) / 2 : 1 + (int64_t)na * na;
  const int li = P->list_of[cls_of[family]];
  const int64_t n = li >= 0 ? P->lists[li].n : 0;
  if (rows) *rows = nrow;
  if (n_A) *n_A = n;
  if (!table && !strings) return E2_OK;
  if (!in || !in->h || !in->B_c || !in->c) return E2_ERR_INVALID_ARG;
  if (P->d.L_extra > 0 && (!in->B_x || !in->w_x)) return E2_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < P->ws_bytes || ((uintptr_t)workspace & 255)) return E2_ERR_WORKSPACE;
  if (n == 0) return E2_OK;
  cudaStream_t st = (cudaStream_t)stream_;
  unsigned char* ws = (unsigned char*)workspace;
  cudaGetLastError();
  g_launches = 0;
  if (setup_common(P, in, ws, st) != E2_OK) return E2_ERR_CUDA;
  const DevList LP = dev_list(P, P->listP, ws);
  const Tabs T = tables(P, ws, root);
  build_tables(P, ws, st, (const double2*)in->c + (int64_t)root * LP.n, T, true);
  const double2* src[5] = {T.DT, T.DTD, T.DTU, T.DTDUD, T.DTDU};
  // rows beyond nrow are padding: the first nrow rows of [Kp][n] are contiguous
  if (table && cudaMemcpyAsync(table, src[family], 16 * (size_t)nrow * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return E2_ERR_CUDA;
  if (strings && cudaMemcpyAsync(strings, dev_list(P, li, ws).str, 8 * (size_t)n, cudaMemcpyDeviceToDevice, st) !=
                     cudaSuccess)
    return E2_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? E2_OK : E2_ERR_CUDA;
}

e2_status e2_probe_couplings(e2_problem* P, const e2_inputs* in, void* workspace, size_t workspace_bytes,
                             void* stream_, int root, int cls, int64_t tile_m, int64_t tile_n, double* V, double* D,
                             int64_t* shape) {
  if (!P || root < 0 || root >= P->d.n_roots || cls < 0 || cls >= E2_NCLASS) return E2_ERR_INVALID_ARG;
  const bool dense = cls == 2 || cls == 5 || cls == 7 || cls == 4 || cls == 6;
  const bool gather = cls == 0 || cls == 1 || cls == 3;
  if ((!dense && !gather) || P->part_cnt[cls] == 0) return E2_ERR_UNSUPPORTED;
  const int64_t nA = P->lists[P->list_of[cls]].n;
  if (shape) {
    shape[0] = dense ? 64 : (cls == 1 ? P->nvc : cls == 3 ? P->ncc : 1);
    shape[1] = dense ? 64 : nA;
  }
  if (!V && !D) return E2_OK;
  if (!in || !in->h || !in->B_c || !in->c || !V || !D) return E2_ERR_INVALID_ARG;
  if (P->d.L_extra > 0 && (!in->B_x || !in->w_x)) return E2_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < P->ws_bytes || ((uintptr_t)workspace & 255)) return E2_ERR_WORKSPACE;
  const DevList L = dev_list(P, P->list_of[cls], (unsigned char*)workspace);
  const int64_t rt = (P->M[cls] + 63) / 64;
  const int64_t nct = P->use_cols[cls] ? P->cplan[cls].tiles : (L.n + 63) / 64;
  if (dense && (tile_m < 0 || tile_m >= rt || tile_n < 0 || tile_n >= nct)) return E2_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream_;
  unsigned char* ws = (unsigned char*)workspace;
  cudaGetLastError();
  g_launches = 0;
  if (setup_common(P, in, ws, st) != E2_OK) return E2_ERR_CUDA;
  setup_classes(P, ws, st);
  const DevList LP = dev_list(P, P->listP, ws);
  const double2* c = (const double2*)in->c + (int64_t)root * LP.n;
  prepare_root(P, ws, st, c, root);
  Ctx X = ctx(P, ws);
  Tabs T = tables(P, ws, root);
  const double b = P->d.level_shift_b;
  double* part = (double*)(ws + P->o_part) + P->part_off[root * E2_NCLASS + cls];
  if (dense) {
    const double2* Dfor[E2_NCLASS] = {nullptr, nullptr, T.DTU, nullptr, T.DTDU, T.DT, T.DTDUD, T.DTD, nullptr};
    cudaMemsetAsync(V, 0, 16 * 64 * 64, st);
    cudaMemsetAsync(D, 0, 8 * 64 * 64, st);
    AdjOut adj{};
    adj.probeV = (double2*)V;
    adj.probeD = D;
    (k_class_probe<<<1, 256, 0, st>>>((const double2*)(ws + P->o_W[cls]), Dfor[cls], P->M[cls], L.n, P->Kp[cls],
                                      (const RowInfo*)(ws + P->o_rows[cls]), L.U, L.eA, X.E0p + root, b,
                                      part + tile_n * rt + tile_m, adj, col_tiles(P, ws, root, cls), tile_m, tile_n,
                                      nct),
     ++g_launches);
  } else {
    DevList Lc[E2_NCLASS];
    for (int k = 0; k < E2_NCLASS; ++k) Lc[k] = dev_list(P, P->list_of[k], ws);
    if (cls == 1)
      (k_class01<<<dim3(blocks(Lc[1].n), (unsigned)P->nvc), 256, 0, st>>>(
           Lc[1], Lc[5], Lc[2], P->das, X.sp, X.binom, T.DT, T.DTU, (const double2*)(ws + P->o_X01), X.f, X.epsh,
           X.E0p + root, b, part, nullptr, (double2*)V, D, 0),
       ++g_launches);
    else if (cls == 3)
      (k_class10<<<dim3(blocks(Lc[3].n), (unsigned)P->ncc), 256, 0, st>>>(
           Lc[3], Lc[7], Lc[5], P->das, X.sp, X.binom, T.DTD, T.DT, (const double2*)(ws + P->o_X10), X.f, X.epsh,
           X.E0p + root, b, part, nullptr, (double2*)V, D, 0),
       ++g_launches);
    else
      (k_class00<<<blocks(Lc[0].n), 256, 0, st>>>(Lc[0], Lc[4], Lc[2], P->das, X.sp, X.binom, T.DTDU, T.DTU,
                                                  (const double2*)(ws + P->o_X00), X.f, X.E0p + root, b, part,
                                                  nullptr, (double2*)V, D, 0),
       ++g_launches);
  }
  return cudaGetLastError() == cudaSuccess ? E2_OK : E2_ERR_CUDA;
}

e2_status e2_form_integrals(e2_problem* P, const e2_inputs* in, void* workspace, size_t workspace_bytes,
                            void* stream_) {
  if (!P || !in || !in->h || !in->B_c) return E2_ERR_INVALID_ARG;
  if (P->d.L_extra > 0 && (!in->B_x || !in->w_x)) return E2_ERR_INVALID_ARG;
  if (!std::isfinite(in->lambda)) return E2_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < P->ws_bytes || ((uintptr_t)workspace & 255)) return E2_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream_;
  unsigned char* ws = (unsigned char*)workspace;
  cudaGetLastError();
  g_launches = 0;
  if (setup_common(P, in, ws, st) != E2_OK) return E2_ERR_CUDA;
  setup_classes(P, ws, st);
  P->launches = g_launches;
  return cudaGetLastError() == cudaSuccess ? E2_OK : E2_ERR_CUDA;
}

e2_status e2_denominator_histogram(e2_problem* P, const e2_inputs* in, void* workspace, size_t workspace_bytes,
                                   void* stream_, int root, unsigned long long* hist) {
  if (!P || !in || !in->h || !in->B_c || !in->c || !hist) return E2_ERR_INVALID_ARG;
  if (P->d.L_extra > 0 && (!in->B_x || !in->w_x)) return E2_ERR_INVALID_ARG;
  if (root < 0 || root >= P->d.n_roots) return E2_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < P->ws_bytes || ((uintptr_t)workspace & 255)) return E2_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream_;
  unsigned char* ws = (unsigned char*)workspace;
  cudaGetLastError();
  g_launches = 0;
  if (setup_common(P, in, ws, st) != E2_OK) return E2_ERR_CUDA;
  setup_classes(P, ws, st);
  const DevList LP = dev_list(P, P->listP, ws);
  prepare_root(P, ws, st, (const double2*)in->c + (int64_t)root * LP.n, root);
  Ctx X = ctx(P, ws);
  cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * E2_NCLASS * E2_DHIST, st);
  for (int cls = 0; cls < E2_NCLASS; ++cls) {
    if (P->part_cnt[cls] == 0) continue;
    const DevList L = dev_list(P, P->list_of[cls], ws);
    dim3 grid((unsigned)P->M[cls], (unsigned)((L.n + 4095) / 4096));
    (k_dhist<<<grid, 256, 0, st>>>(cls, X.sp, L, X.epsh, X.G, X.E0p + root, hist + cls * E2_DHIST), ++g_launches);
  }
  return cudaGetLastError() == cudaSuccess ? E2_OK : E2_ERR_CUDA;
}

e2_status e2_prepare_roots(e2_problem* P, const e2_inputs* in, void* workspace, size_t workspace_bytes,
                           void* stream_) {
  if (!P || !in || !in->h || !in->B_c || !in->c) return E2_ERR_INVALID_ARG;
  if (P->d.L_extra > 0 && (!in->B_x || !in->w_x)) return E2_ERR_INVALID_ARG;
  if (!std::isfinite(in->lambda)) return E2_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < P->ws_bytes || ((uintptr_t)workspace & 255)) return E2_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream_;
  unsigned char* ws = (unsigned char*)workspace;
  cudaGetLastError();
  g_launches = 0;
  if (setup_common(P, in, ws, st) != E2_OK) return E2_ERR_CUDA;
  const DevList LP = dev_list(P, P->listP, ws);
  for (int r = 0; r < P->d.n_roots; ++r) prepare_root(P, ws, st, (const double2*)in->c + (int64_t)r * LP.n, r);
  return cudaGetLastError() == cudaSuccess ? E2_OK : E2_ERR_CUDA;
}

e2_status e2_set_shard(e2_problem* P, int rank, int n_ranks) {
  if (!P || n_ranks < 1 || rank < 0 || rank >= n_ranks) return E2_ERR_INVALID_ARG;
  P->shard_rank = rank;
  P->shard_n = n_ranks;
  return E2_OK;
}

e2_status e2_shard_units(const e2_problem* P, int cls, int64_t* units, int64_t* first, int64_t* end) {
  if (!P || cls < 0 || cls >= E2_NCLASS) return E2_ERR_INVALID_ARG;
  int64_t u0, u1;
  shard_range(P, cls, u0, u1);
  if (units) *units = shard_units(P, cls);
  if (first) *first = u0;
  if (end) *end = u1;
  return E2_OK;
}

e2_status e2_shard_buffers(const e2_problem* P, void* workspace, double** partials, int64_t* n_partials,
                           int64_t** min_keys, int64_t* n_keys) {
  if (!P || !workspace) return E2_ERR_INVALID_ARG;
  unsigned char* ws = (unsigned char*)workspace;
  if (partials) *partials = (double*)(ws + P->o_part);
  if (n_partials) *n_partials = part_total(P);
  if (min_keys) *min_keys = (int64_t*)dmin_slot(P, ws, 0, 0);
  if (n_keys) *n_keys = (int64_t)P->d.n_roots * E2_NCLASS;
  return E2_OK;
}

e2_status e2_reduce(e2_problem* P, void* workspace, size_t workspace_bytes, void* stream_, double* E2,
                    double* E2_class, double* E0) {
  if (!P || !E2) return E2_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < P->ws_bytes || ((uintptr_t)workspace & 255)) return E2_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream_;
  unsigned char* ws = (unsigned char*)workspace;
  cudaGetLastError();
  g_launches = 0;
  cudaMemsetAsync(status_word(P, ws), 0, sizeof(unsigned long long), st);  // flags again from the summed partials
  launch_reduce(P, ws, st, E2, E2_class, E0);
  return cudaGetLastError() == cudaSuccess ? E2_OK : E2_ERR_CUDA;
}

e2_status e2_query_status(const e2_problem* P, const void* workspace, void* stream_, uint32_t* flags,
                          double* min_abs_D) {
  if (!P) return E2_ERR_INVALID_ARG;
  const unsigned char* ws = (const unsigned char*)workspace;
  if (!ws) {
    ws = (const unsigned char*)noalloc_scratch();
    if (!ws) return E2_ERR_CUDA;
  }
  const int R = P->d.n_roots;
  std::vector<unsigned long long> h((size_t)1 + (size_t)R * E2_NCLASS);
  cudaStream_t st = (cudaStream_t)stream_;
  if (cudaMemcpyAsync(h.data(), ws + P->o_status, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return E2_ERR_CUDA;
  if (flags) *flags = (uint32_t)h[0];
  if (min_abs_D)
    for (int k = 0; k < R * E2_NCLASS; ++k) {
      const unsigned long long key = h[1 + k];
      double v;
      std::memcpy(&v, &key, sizeof v);
      min_abs_D[k] = key >= 0x7FF0000000000000ULL ? INFINITY : v;
    }
  if (h[0] & ST_NONFINITE) return E2_ERR_NONFINITE;
  if (h[0] & ST_INTRUDER) return E2_ERR_INTRUDER;
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
    *columns = (P->use_cols[cls] && !P->use_oz[cls])
                   ? (const int32_t*)((const unsigned char*)workspace + P->cplan[cls].o_perm)
                   : nullptr;
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
                                           part + P->part_off[c], AdjOut{}, col_tiles(P, ws, 0, c), nullptr,
                                           (int64_t)grid.x, 0);
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

// Key of a problem's tuning entry: every plan input that changes the class
// shapes (spinor counts, partition, frozen spinors, factor counts, roots,
// class mask), as one text line.
static std::string tuning_key(const e2_problem* P) {
  const e2_desc& d = P->d;
  std::string k = "e2tune1 " + std::to_string(d.n_core) + " " + std::to_string(d.n_active) + " " +
                  std::to_string(d.n_virt) + " " + std::to_string(d.n_elec) + " das";
  for (int s = 0; s < d.n_das; ++s)
    k += " " + std::to_string(P->das_size[s]) + ":" + std::to_string(P->das_min[s]) + ":" + std::to_string(P->das_max[s]);
  k += " ham " + std::to_string(d.ham) + " L " + std::to_string(d.L_coulomb) + " " + std::to_string(d.L_extra) +
       " roots " + std::to_string(d.n_roots) + " mask " + std::to_string(d.class_mask) + " frozen ";
  for (uint8_t f : P->frozen) k += f ? '1' : '0';
  return k;
}

e2_status e2_tuning_save(const e2_problem* P, const char* path) {
  if (!P || !path) return E2_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "a");
  if (!f) return E2_ERR_INVALID_ARG;
  std::fprintf(f, "%s |", tuning_key(P).c_str());
  for (int c = 0; c < E2_NCLASS; ++c) std::fprintf(f, " %d", P->use_cols[c] ? 1 : 0);
  std::fprintf(f, "\n");
  const bool ok = std::fclose(f) == 0;
  return ok ? E2_OK : E2_ERR_INVALID_ARG;
}

e2_status e2_tuning_load(e2_problem* P, const char* path) {
  if (!P || !path) return E2_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "r");
  if (!f) return E2_ERR_UNSUPPORTED;
  const std::string key = tuning_key(P) + " |";
  std::string line, hit;
  int ch;
  while (true) {  // the last matching entry wins
    line.clear();
    while ((ch = std::fgetc(f)) != EOF && ch != '\n') line.push_back((char)ch);
    if (line.compare(0, key.size(), key) == 0) hit = line.substr(key.size());
    if (ch == EOF) break;
  }
  std::fclose(f);
  if (hit.empty()) return E2_ERR_UNSUPPORTED;
  int v[E2_NCLASS];
  if (std::sscanf(hit.c_str(), "%d %d %d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6], &v[7],
                  &v[8]) != E2_NCLASS)
    return E2_ERR_UNSUPPORTED;
  for (int c = 0; c < E2_NCLASS; ++c) P->use_cols[c] = v[c] && P->cplan[c].built;
  return E2_OK;
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

}  // extern "C"

// ------------------------------------------------------------------ fixed scratch variant

// Scratch for e2_forward_noalloc, compiled into the library: every device
// that loads it holds these bytes until the process exits.  Nothing in the
// forward layout needs to start at zero (every buffer is fully written before
// it is read; the status word is cleared by the call itself), so calls do not
// clear it; consecutive calls simply overwrite it.
static __device__ __align__(256) unsigned char e2_static_scratch[E2_STATIC_SCRATCH_BYTES];

namespace e2 {
// Device address of the scratch array on the current device.  Looked up on
// every call, with that device current: the host-side symbol is only a
// stand-in, and an address kept from an earlier context would not survive a
// device reset.
void* noalloc_scratch() {
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, e2_static_scratch) != cudaSuccess) return nullptr;
  return ptr;
}
}  // namespace e2

extern "C" e2_status e2_forward_noalloc(e2_problem* P, const e2_inputs* in, void* stream, double* E2,
                                        double* E2_class, double* E0) {
  if (!P) return E2_ERR_INVALID_ARG;
  if (P->ws_bytes > (size_t)E2_STATIC_SCRATCH_BYTES) return E2_ERR_WORKSPACE;  // before any GPU call
  void* ptr = noalloc_scratch();
  if (!ptr) return E2_ERR_CUDA;
  return e2_forward(P, in, ptr, (size_t)E2_STATIC_SCRATCH_BYTES, stream, E2, E2_class, E0);
}
