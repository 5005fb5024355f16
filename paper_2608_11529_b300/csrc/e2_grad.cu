// C ABI: the adjoint pass (e2_backward): E2 and its gradients with respect
// to h, the factors, c and lambda, V recomputed tile by tile.
#include "e2_host.h"


using namespace e2;

extern "C" {

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
  if (P->shard_n > 1) return E2_ERR_UNSUPPORTED;  // the adjoint runs unsharded
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
  if (want_B) {
    cudaMemsetAsync(Ge, 0, 8 * (size_t)std::max(nx, 1) * std::max(nx, 1), st);
    cudaMemsetAsync(Gea, 0, 8 * (size_t)std::max(nx, 1) * std::max(na, 1), st);
    cudaMemsetAsync(Ntt, 0, 8 * (size_t)na * na, st);
    cudaMemsetAsync(Gt, 0, 16 * (size_t)npair * npair, st);
  }
  // denominators of rows with external spinors: with z_e the signed incidence
  // of row e (+1 on its particles, -1 on its holes),
  //   Ge[x][y] += sum_e hs[e] z_e[x] z_e[y],  Gea[x][t] += sum_e z_e[x] hocc[e][t],
  // formed from marginals of hs and hocc over the (hole tuple, particle tuple)
  // structure of the class's rows.
  auto zpair = [&](int cls, const double* hs, const double* hocc) {
    const int ncc = P->ncc, nvc = P->nvc;
    const int64_t ncp = pairs(ncc), nvp = pairs(nvc);
    int kh = 0, kp = 0;
    switch (cls) {
      case 2: kp = 2; break;
      case 5: kh = 1; kp = 2; break;
      case 7: kh = 2; kp = 1; break;
      case 4: kh = 1; kp = 1; break;
      case 6: kh = 2; break;
      case 1: kp = 1; break;
      case 3: kh = 1; break;
      case 8: kh = 2; kp = 2; break;
      default: return;
    }
    const int64_t nh = kh == 0 ? 1 : kh == 1 ? ncc : ncp, np_ = kp == 0 ? 1 : kp == 1 ? nvc : nvp;
    if (nh == 0 || np_ == 0) return;
    double* Sp = Zm;              // [np]      sum over holes
    double* Sh = Sp + np_;        // [nh]      sum over particles
    double* Spo = Sh + nh;        // [np][na]  hocc summed over holes
    double* Sho = Spo + np_ * na; // [nh][na]  hocc summed over particles
    double* Cr = Sho + nh * na;   // [nh][nvc] per hole tuple, summed over the particle tuples holding a
    const int64_t dg = nx + 1;    // stride of Ge's diagonal
    (k_colsum<<<blocks(np_), 256, 0, st>>>(hs, nh, np_, 0, Sp), ++g_launches);
    if (np_ >= 256)
      (k_rowsum_wide<<<(unsigned)nh, 256, 0, st>>>(hs, np_, 0, Sh), ++g_launches);
    else
      (k_rowsum<<<blocks(nh), 256, 0, st>>>(hs, nh, np_, 0, Sh), ++g_launches);
    if (kp) {
      (k_tmarg<<<blocks(nvc), 256, 0, st>>>(Sp, 1, np_, 1, kp, nvc, 1.0, 1, Ge + ncc * dg, 0, dg, 0), ++g_launches);
      if (kp == 2)
        (k_pairplace<<<blocks((int64_t)nvc * nvc), 256, 0, st>>>(Sp, nvc, Ge + (int64_t)ncc * nx + ncc, nx),
         ++g_launches);
      (k_colsum<<<blocks(np_ * na), 256, 0, st>>>(hocc, nh, np_ * na, 0, Spo), ++g_launches);
      (k_tmarg<<<blocks((int64_t)nvc * na), 256, 0, st>>>(Spo, 1, np_, na, kp, nvc, 1.0, 1, Gea + (int64_t)ncc * na,
                                                         0, na, 1), ++g_launches);
    }
    if (kh) {
      (k_tmarg<<<blocks(ncc), 256, 0, st>>>(Sh, 1, nh, 1, kh, ncc, 1.0, 1, Ge, 0, dg, 0), ++g_launches);
      if (kh == 2) (k_pairplace<<<blocks((int64_t)ncc * ncc), 256, 0, st>>>(Sh, ncc, Ge, nx), ++g_launches);
      (k_midsum<<<(unsigned)nh, 256, 0, st>>>(hocc, np_, na, Sho), ++g_launches);
      (k_tmarg<<<blocks((int64_t)ncc * na), 256, 0, st>>>(Sho, 1, nh, na, kh, ncc, -1.0, 1, Gea, 0, na, 1),
       ++g_launches);
    }
    if (kh && kp) {  // hole-particle entries, both orders
      (k_tmarg<<<blocks(nh * nvc), 256, 0, st>>>(hs, nh, np_, 1, kp, nvc, 1.0, 0, Cr, nvc, 1, 0), ++g_launches);
      (k_tmarg<<<blocks((int64_t)ncc * nvc), 256, 0, st>>>(Cr, 1, nh, nvc, kh, ncc, -1.0, 1, Ge + ncc, 0, nx, 1),
       ++g_launches);
      (k_tmarg<<<blocks((int64_t)ncc * nvc), 256, 0, st>>>(Cr, 1, nh, nvc, kh, ncc, -1.0, 1, Ge + (int64_t)ncc * nx,
                                                          0, 1, nx), ++g_launches);
    }
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
          if (P->use_oz[cls]) {
            launch_class_oz(st, cls, oz_operands(P, ws, r, cls), P->M[cls], Lc[cls].n,
                            (const RowInfo*)(ws + P->o_rows[cls]), X.E0p + r, b, poff(cls), dmin_slot(P, ws, r, cls));
            continue;
          }
          dim3 grid((unsigned)((P->M[cls] + 63) / 64), (unsigned)((Lc[cls].n + 63) / 64));
          (k_class_gemm<<<grid, 256, 0, st>>>((const double2*)(ws + P->o_W[cls]), Df[cls], P->M[cls], Lc[cls].n,
                                              P->Kp[cls], (const RowInfo*)(ws + P->o_rows[cls]), Lc[cls].U, Lc[cls].eA,
                                              X.E0p + r, b, poff(cls), AdjOut{}, col_tiles(P, ws, r, cls),
                                              dmin_slot(P, ws, r, cls), (int64_t)grid.x, 0), ++g_launches);
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
      // (on the sliced GEMM the products take plain columns: their tensor work
      // no longer dominates)
      const bool slg = P->use_oz_adj;
      const bool tiled = !slg && P->use_cols[cls] && P->cplan[cls].gran == 8;
      const ColPlan& cp = P->cplan[cls];
      const ColTiles ctl = col_tiles(P, ws, r, cls);
      // E2 of a class on the sliced contraction: the forward's own kernel, so
      // that the energies equal e2_forward's bit for bit
      if (E2 && P->use_oz[cls])
        launch_class_oz(st, cls, oz_operands(P, ws, r, cls), M, N, (const RowInfo*)(ws + P->o_rows[cls]), X.E0p + r, b,
                        poff(cls), dmin_slot(P, ws, r, cls));
      double* part_adj = P->use_oz[cls] ? nullptr : poff(cls);
      for (int64_t m0 = 0; m0 < M; m0 += P->chunk_rows[cls]) {
        const int64_t Mc = std::min<int64_t>(P->chunk_rows[cls], M - m0);
        // float-float amplitudes when the sliced products will read them: the
        // class on the sliced contraction, its products on the sliced GEMM, and
        // their slices within the scratch
        const bool tdf = P->use_oz[cls] && slg &&
                         zgemm_sliced_bytes(N, Kp, Mc, OZ_ADJ_S) <= P->bOz_bytes &&
                         (!want_B || zgemm_sliced_bytes(Mc, Kp, N, OZ_ADJ_S) <= P->bOz_bytes);
        AdjOut adj{(double2*)B(P->o_bT), want_B ? (double*)B(P->o_bHm) : nullptr, (double*)B(P->o_bHrow),
                   (double*)B(P->o_bHcol), (double*)B(P->o_bScalT), m0, Mc, s, g1, part_adj, rt, tdf ? 1 : 0};
        // FP64 products over column tiles read T (and Hm) in tile column order
        const bool tile_order = tiled && !P->use_oz[cls];
        adj.t_tile = tile_order ? 1 : 0;
        adj.t_ld = tile_order ? 64 * cp.tiles : 0;
        const int32_t* tperm = tile_order ? ctl.perm : nullptr;
        dim3 grid((unsigned)((Mc + 63) / 64), (unsigned)ct);
        if (P->use_oz[cls])  // the sliced contraction in its adjoint mode (plain columns)
          launch_class_oz_adj(st, cls, oz_operands(P, ws, r, cls), M, N, (const RowInfo*)(ws + P->o_rows[cls]),
                              X.E0p + r, b, adj);
        else
          (k_class_gemm<<<grid, 256, 0, st>>>(W, Dfor[cls], M, N, (int)Kp, (const RowInfo*)(ws + P->o_rows[cls]), L.U,
                                              L.eA, X.E0p + r, b, nullptr, adj, col_tiles(P, ws, r, cls),
                                              dmin_slot(P, ws, r, cls), (int64_t)grid.x, 0),
           ++g_launches);
        // per-tile sums of this chunk: row sums of eta, column sums per row tile, the scalars
        {
          const int64_t rtc = (Mc + 63) / 64;
          (k_rowsum<<<blocks(Mc), 256, 0, st>>>(adj.Hrow, Mc, ct, 0, hsum + m0), ++g_launches);
          (k_colsum<<<blocks(N), 256, 0, st>>>(adj.Hcol, rtc, N, m0 > 0, hA), ++g_launches);
          (k_scalsum<<<1, 256, 0, st>>>(adj.scal, rtc * ct, scal), ++g_launches);
        }
        // Gamma_D[x][A] += sum_e W[e][x] conj(T[e][A]) (split over the rows of the chunk)
        if (tiled)
          zgemm_gd_tiles(st, cp, ctl, W + m0 * Kp, (int)Kp, adj.T, N, Mc, (double2*)B(P->o_bGDc), m0 > 0, 1, adj.t_ld);
        else if (slg && zgemm_sliced(st, N, Kp, Mc, adj.T, 1, N, 1, W + m0 * Kp, Kp, 1, 0, GDfor[cls], 1, N, 1, -1,
                                     (unsigned char*)B(P->o_bOz), P->bOz_bytes, 0, false, OZ_ADJ_S, tdf))
          ;  // Gamma_D^T = conj(T)^T W: T is the row operand (sliced without duplication)
        else if (Kp >= 64)
          zgemm(st, Kp, N, Mc, W + m0 * Kp, 1, Kp, 0, adj.T, N, 1, 1, GDfor[cls], N, 1, 1, 64);
        else
          zgemm(st, N, Kp, Mc, adj.T, 1, N, 1, W + m0 * Kp, Kp, 1, 0, GDfor[cls], 1, N, 1, 16);
        if (cls == 4)
          (k_rowdot<<<(unsigned)Mc, 256, 0, st>>>(adj.T, T.DTDU, N, (double2*)B(P->o_bRowdot) + m0, tperm, adj.t_ld),
           ++g_launches);
        if (want_B) {  // Gamma_W = conj(T) D^T and the per-row occupation sums of eta
          double2* GW = (double2*)B(P->o_bGW[cls]) + m0 * Kp;
          if (tiled) {  // per tile over its compacted rows, then summed per table row in tile order
            launch_gw_tiles(cp.pbn, Mc, cp.maxklen, cp.tiles, st, ctl, adj.T, N, cp.krows, (double2*)B(P->o_bGWc), 1,
                            adj.t_ld);
            (k_gw_reduce<<<blocks(Mc * Kp), 256, 0, st>>>(ctl.tdesc, (const int32_t*)(ws + cp.o_pos), cp.tiles,
                                                         (int)Kp, (const double2*)B(P->o_bGWc), cp.krows, Mc, GW,
                                                         (int)Kp, Kp), ++g_launches);
          } else if (!(slg && zgemm_sliced(st, Mc, Kp, N, adj.T, N, 1, 1, Dfor[cls], 1, N, 0, GW, Kp, 1, 0, -1,
                                           (unsigned char*)B(P->o_bOz), P->bOz_bytes, 0, false, OZ_ADJ_S,
                                           tdf))) {
            zgemm(st, Mc, Kp, N, adj.T, N, 1, 1, Dfor[cls], 1, N, 0, GW, Kp, 1, 0, Kp >= 64 ? 64 : 16);
          }
          if (P->use_oz[cls])  // eta came as float-float pairs from the sliced adjoint
            launch_hocc_df(st, (const float2*)adj.Hm, L, na, Mc, Hocc + m0 * na);
          else
            (k_hocc<<<(unsigned)Mc, 256, 0, st>>>(adj.Hm, L, na, Hocc + m0 * na, tperm, adj.t_ld), ++g_launches);
        }
      }
      if (tiled)
        (k_gd_scatter<<<(unsigned)cp.tiles, 256, 0, st>>>(ctl, (const double2*)B(P->o_bGDc), N, GDfor[cls]),
         ++g_launches);
      if (cls == 4) (k_fock11<<<blocks(M), 256, 0, st>>>((const double2*)B(P->o_bRowdot), X.sp, Gf), ++g_launches);
      (k_xmarg<<<P->nx, 256, 0, st>>>((const RowInfo*)(ws + P->o_rows[cls]), hsum, M, P->nx, Nx), ++g_launches);
      (k_amarg<<<na, 256, 0, st>>>(L, hA, Nt), ++g_launches);
      if (want_B) {
        zpair(cls, hsum, Hocc);
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
      const int64_t nyb = (int64_t)P->nvb * (P->nvb + 1) / 2;
      c22 = (double*)B(P->o_bC22);
      if (E2 && P->use_oz[8]) {
        const HostList& H8 = P->lists[P->list_of[8]];
        launch_class22_df(st, L, X.sp, (const float2*)(ws + H8.o_eAdf), (const float2*)(ws + H8.o_Udf), c,
                          (const double*)(ws + P->o_G22), X.epsh, X.G, X.E0p + r, b, P->nvb, P->ncp, poff(8),
                          dmin_slot(P, ws, r, 8));
      }
      // chunks of core pairs: partials of one chunk, reduced before the next
      for (int z0 = 0; z0 < (int)P->ncp; z0 += P->z22_chunk) {
        const int zc = (int)std::min<int64_t>(P->z22_chunk, P->ncp - z0);
        const int64_t yz = nyb * zc;
        dim3 grid(blocks(L.n), (unsigned)nyb, (unsigned)zc);
        // E2 from the forward's float-float kernel when the class uses it (then
        // the adjoint kernel writes no partials)
        (k_class22_bwd<<<grid, 256, 0, st>>>(L, X.sp, c, (const double*)(ws + P->o_G22), X.epsh, X.G, X.E0p + r, b,
                                             P->nvb, s, g1, (double*)B(P->o_bC22p), (double*)B(P->o_bH22p),
                                             (double*)B(P->o_bV22), P->use_oz[8] ? nullptr : poff(8), z0),
         ++g_launches);
        (k_colsum<<<blocks(L.n), 256, 0, st>>>((const double*)B(P->o_bC22p), yz, L.n, z0 > 0, c22), ++g_launches);
        (k_colsum<<<blocks(L.n), 256, 0, st>>>((const double*)B(P->o_bH22p), yz, L.n, z0 > 0, hA), ++g_launches);
        (k_class22_marg<<<(unsigned)(P->nvc + P->ncc + 1), 256, 0, st>>>((const double*)B(P->o_bV22),
                                                                     (int)blocks(L.n), P->nvb, zc, z0, X.sp, Nx,
                                                                     scal), ++g_launches);
      }
      (k_amarg<<<na, 256, 0, st>>>(L, hA, Nt), ++g_launches);
      if (want_B) {
        const int64_t M22 = P->ncp * P->nvp;
        double* hs22 = (double*)B(P->o_bHs22);
        double* P22 = (double*)B(P->o_bP22);
        const HostList& H8 = P->lists[P->list_of[8]];
        if (P->use_oz_adj && H8.df) {  // float-float per-row sums
          float2* c2 = (float2*)B(P->o_bC2);
          (k_c2df<<<blocks(L.n), 256, 0, st>>>(c, L.n, g1, c2), ++g_launches);
          launch_class22_rows_df(st, L, X.sp, (const float2*)(ws + H8.o_eAdf), (const float2*)(ws + H8.o_Udf), c2,
                                 (const double*)(ws + P->o_G22), X.epsh, X.G, X.E0p + r, b, s, M22, hs22, Hocc, P22);
        } else {
          (k_class22_rows<<<(unsigned)M22, occ_threads(na), occ_smem(na), st>>>(
               L, X.sp, c, (const double*)(ws + P->o_G22), X.epsh, X.G, X.E0p + r, b, s, g1, hs22, Hocc, P22),
           ++g_launches);
        }
        zpair(8, hs22, Hocc);
        (k_ntt<<<na * na, 256, 0, st>>>(L, hA, na, Ntt), ++g_launches);
        const int Lt = d.L_coulomb + d.L_extra;
        (k_integrals<<<blocks(M22), 256, 0, st>>>(INT_G22C, X.sp, X.Bo, X.wt, Lt, X.f, P->ncp, (int)P->nvp,
                                                  (int)P->nvp, B(P->o_bG22c)), ++g_launches);
        if (P->ext_das)  // rows outside Q take no part in the factor gradient
          (k_mask22<<<blocks(M22), 256, 0, st>>>(B(P->o_bG22c), P->ncp, P->nvp, X.sp, 1), ++g_launches);
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
        (k_hocc<<<(unsigned)nrow, 256, 0, st>>>(Hg, L, na, Hocc, nullptr, 0), ++g_launches);
        zpair(cls, hsum, Hocc);
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
        const bool tl = !P->use_oz_adj && tcls >= 0 && P->use_cols[tcls];
        unsigned char* oz = (unsigned char*)B(P->o_bOz);
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
          else if (!(P->use_oz_adj &&  // Gamma_D^T = Tsh^T X: Tsh is the row operand
                     zgemm_sliced(st, nb, nx_, k, Tsh, 1, nb, 0, Xr, nx_, 1, 0, GD, 1, nb, 1, -1, oz, P->bOz_bytes, 0, false, OZ_ADJ_S)))
            zgemm(st, nx_, nb, k, Xr, 1, nx_, 0, Tsh, nb, 1, 0, GD, nb, 1, 1);
          if (want_B) {
            double2* GXr = GX + (int64_t)r0 * S * nx_;
            if (tl) {
              launch_gw_tiles(cpt.pbn, k, cpt.maxklen, cpt.tiles, st, ctt, Tsh, nb, cpt.krows,
                              (double2*)B(P->o_bGWc), 0, 0);
              // written, not accumulated: gx_beta is set only for class (0,0),
              // one row, whose target is still zero here
              (k_gw_reduce<<<blocks(k * nx_), 256, 0, st>>>(ctt.tdesc, (const int32_t*)(ws + cpt.o_pos), cpt.tiles,
                                                           P->Kp[tcls], (const double2*)B(P->o_bGWc), cpt.krows, k,
                                                           GXr, nx_, nx_), ++g_launches);
            } else if (!(P->use_oz_adj && zgemm_sliced(st, k, nx_, nb, Tsh, nb, 1, 0, D, 1, nb, 0, GXr, nx_, 1,
                                                       gx_beta, -1, oz, P->bOz_bytes, 0, false, OZ_ADJ_S))) {
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
    if (!(P->use_oz_adj && zgemm_sliced(st, Lt, npair, npair, X.Bo, npair, 1, 0, Gh, 1, npair, 0, Cs, npair, 1, 0, -1,
                                        (unsigned char*)B(P->o_bOz), P->bOz_bytes, 0, false, OZ_ADJ_S)))
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

}  // extern "C"
