// Kernel entry points (defined in e2_kernels.cu and e2_adjoint.cu), launched by the host units.
#pragma once
#include "e2_common.cuh"

namespace e2 {

__global__ void k_binom(int64_t* tab);
__global__ void k_extract(const double2* Bc, const double2* Bx, const double* wx, double lambda, int Lc, int Lx, int n,
                          int nocc, double2* Bo, double* wt, double* dg);
__global__ void k_G(const double2* Bc, const double2* Bx, const double* wt, const double* dg, int Lc, int Lx, int n,
                    double* G);
__global__ void k_fock(const double2* h, const double2* Bo, const double* wt, const double* dg, int L, int n, int nocc,
                       int ncore, double2* f);
__global__ void k_scalars(const double2* h, const double* G, int n, int ncore, double* epsh, double* EO);
__global__ void k_unrank(DevList Ls, DevDas das, const int64_t* binom);
__global__ void k_eA(DevList Ls, const double* epsh, const double* G, int n, int a0);
__global__ void k_U(DevList Ls, DevSpace sp, const double* G);
__global__ void k_integrals(int mode, DevSpace sp, const double2* Bo, const double* wt, int L, const double2* f,
                            int64_t rows, int cols, int ld, void* out);
__global__ void k_vafactors(DevSpace sp, const double2* Bo, const double* wt, int Lt, double2* Yw, double2* Z);
__global__ void k_xfactors(DevSpace sp, const double2* Bo, const double* wt, int Lt, double2* Ywc, double2* Zaa);
__global__ void k_w12(DevSpace sp, const double2* X, int64_t ldx, int64_t M, int Kp, double2* W);
__global__ void k_x01(DevSpace sp, const double2* X, double2* X01);
__global__ void k_w02(DevSpace sp, const double2* X, int64_t ldx, int b0, int b1, int Kp, double2* W);
__global__ void k_rows(int cls, DevSpace sp, const double* epsh, const double* G, int64_t M, RowInfo* out);
__global__ void k_mask_rows(double2* W, int64_t M, int Kp, const RowInfo* rows);
__global__ void k_mask22(void* g, int64_t ncp, int64_t nvp, DevSpace sp, int cplx);
__global__ void k_dhist(int cls, DevSpace sp, DevList L, const double* epsh, const double* G, const double* E0p,
                        unsigned long long* hist);
__global__ void k_dtable(int fam, DevList Ls, DevList Pl, DevDas das, const int64_t* binom, const double2* c, int Kp,
                         double2* D);
__global__ void k_gram(const double2* Da, const double2* Db, int64_t n, int ny, double2* out);
__global__ void k_e0(const double2* g1, const double2* g2, const double2* f, const double2* X00, DevSpace sp, int ntp,
                     const double* EO, double* E0p, double* E0);
__global__ void k_class_gemm(const double2* W, const double2* D, int64_t M, int64_t N, int Kp, const RowInfo* rows,
                             const double* U, const double* eA, const double* E0p, double b, double* partial, AdjOut adj, ColTiles ctl,
                             unsigned long long* dmin, int64_t rt, int64_t tm0);
__global__ void k_dcompact(const double2* D, int64_t N, ColTiles ctl, double2* Dc);
__global__ void k_class_probe(const double2* W, const double2* D, int64_t M, int64_t N, int Kp, const RowInfo* rows,
                              const double* U, const double* eA, const double* E0p, double b, double* partial,
                              AdjOut adj, ColTiles ctl, int64_t tile_m, int64_t tile_n, int64_t n_tile_n);
__global__ void k_batch(const WorkSeg* segs, int nseg, const GemmJob* gjobs, const SparseJob* sjobs, int64_t total,
                        unsigned long long* counter);
__global__ void k_class22(DevList Ls, DevSpace sp, const double2* c, const double* g2, const double* epsh,
                          const double* G, const double* E0p, double b, int nvb, double* partial,
                          unsigned long long* dmin, int64_t u0);
__global__ void k_class01(DevList L01, DevList L12, DevList L02, DevDas das, DevSpace sp, const int64_t* binom,
                          const double2* DT, const double2* DTU, const double2* X01, const double2* f,
                          const double* epsh, const double* E0p, double b, double* partial,
                          unsigned long long* dmin, double2* probeV,
                          double* probeD, int64_t u0);
__global__ void k_class10(DevList L10, DevList L21, DevList L12, DevDas das, DevSpace sp, const int64_t* binom,
                          const double2* DTD, const double2* DT, const double2* X10, const double2* f,
                          const double* epsh, const double* E0p, double b, double* partial,
                          unsigned long long* dmin, double2* probeV,
                          double* probeD, int64_t u0);
__global__ void k_class00(DevList L00, DevList L11, DevList L02, DevDas das, DevSpace sp, const int64_t* binom,
                          const double2* DTDU, const double2* DTU, const double2* X00, const double2* f,
                          const double* E0p, double b, double* partial, unsigned long long* dmin, double2* probeV,
                          double* probeD, int64_t u0);
__global__ void k_sigma(DevList LP, DevList L11, DevList L02, DevDas das, DevSpace sp, const int64_t* binom,
                        const double2* DTDU, const double2* DTU, const double2* X00, const double2* f, double2* sigma);
__global__ void k_lincomb(const double2* V, int m, int64_t n, const double2* Y, int k, int acc, double2* out);
__global__ void k_residual(double2* r, const double2* x, const double* diag, int64_t n, double theta, double2* d);
__global__ void k_scale(double2* x, int64_t n, double s);
__global__ void k_peak_dmma(double* out, int iters);
__global__ void k_peak_dfma(double* out, int iters);
__global__ void k_reduce(const double* partial, const int64_t* off, const int64_t* cnt, const double2* g1_all,
                         int g1_stride, int n_roots, double* e2c);
__global__ void k_status_init(unsigned long long* status, int n);
__global__ void k_finalize(const double* e2c, int n_roots, double* E2, const double* E0in, double* E0out,
                           unsigned long long* status, double b);

// sliced bf16 contraction (e2_ozaki.cu)
__global__ void k_c2df(const double2* c, int64_t n, const double2* g1, float2* out);
__global__ void k_oz_colmax(const double2* B, int64_t sbk, int64_t sbn, int K, int64_t N, int kchunk,
                            unsigned long long* cmax);
__global__ void k_oz_tables(const double* eA, const double* U, int64_t n, int64_t rows, float2* eAdf, float2* Udf);

// adjoint (e2_adjoint.cu)
__global__ void k_zgemm64(int64_t M, int64_t N, int64_t K, const double2* A, int64_t sam, int64_t sak, int conjA,
                          const double2* B, int64_t sbk, int64_t sbn, int conjB, double2* C, int64_t csm, int64_t csn,
                          int beta, int64_t kseg, int64_t czs, int64_t lower);
__global__ void k_zgemm16(int64_t M, int64_t N, int64_t K, const double2* A, int64_t sam, int64_t sak, int conjA,
                          const double2* B, int64_t sbk, int64_t sbn, int conjB, double2* C, int64_t csm, int64_t csn,
                          int beta, int64_t kseg, int64_t czs, int64_t lower);
__global__ void k_zgemm24(int64_t M, int64_t N, int64_t K, const double2* A, int64_t sam, int64_t sak, int conjA,
                          const double2* B, int64_t sbk, int64_t sbn, int conjB, double2* C, int64_t csm, int64_t csn,
                          int beta, int64_t kseg, int64_t czs, int64_t lower);
// compacted Gamma products of a column-tiled class at product width bn (32, 48, 64, 80)
void launch_gd_tiles(int bn, dim3 grid, cudaStream_t st, const ColTiles& ctl, const double2* W, int Kp,
                     const double2* T, int64_t N, int64_t Mc, double2* GDc, int beta, int64_t kseg, int64_t czs,
                     int conjT, int64_t t_ld);
void launch_gw_tiles(int bn, int64_t Mc, int maxklen, int64_t tiles, cudaStream_t st, const ColTiles& ctl,
                     const double2* T, int64_t N, int64_t krows, double2* GWc, int conjT, int64_t t_ld);
__global__ void k_gd_scatter(ColTiles ctl, const double2* GDc, int64_t N, double2* GD);
__global__ void k_gw_reduce(const int4* tdesc, const int32_t* pos, int64_t tiles, int Kp, const double2* GWc,
                            int64_t krows, int64_t Mc, double2* GW, int nxo, int64_t ldo);
__global__ void k_zacc(const double2* part, int nseg, int64_t ps, int64_t M, int64_t N, double2* C, int64_t csm,
                       int64_t csn, int beta);
__global__ void k_rowsum_wide(const double* in, int64_t ncol, int acc, double* out);
__global__ void k_rowsum(const double* in, int64_t nrow, int64_t ncol, int acc, double* out);
__global__ void k_colsum(const double* in, int64_t nrow, int64_t ncol, int acc, double* out);
__global__ void k_scalsum(const double* in, int64_t n, double* scal_out);
__global__ void k_xmarg(const RowInfo* rows, const double* hsum, int64_t M, int nx, double* Nx);
__global__ void k_amarg(DevList Ls, const double* hA, double* Nt);
__global__ void k_rowdot(const double2* T, const double2* d, int64_t N, double2* out, const int32_t* perm,
                         int64_t ld);
__global__ void k_fock11(const double2* rowdot, DevSpace sp, double2* Gf);
__global__ void k_class22_bwd(DevList Ls, DevSpace sp, const double2* c, const double* g2, const double* epsh,
                              const double* G, const double* E0p, double b, int nvb, double s, const double2* g1,
                              double* cpart, double* hpart, double* vpart, double* part, int z0);
__global__ void k_class22_marg(const double* vpart, int nx_blocks, int nvb, int64_t ncp, int z0, DevSpace sp,
                               double* Nx, double* scal);
__global__ void k_gather_t(int cls, DevList Lx, DevList L12, DevList L02, DevList L21, DevList L11, DevDas das,
                           DevSpace sp, const int64_t* binom, const double2* DT, const double2* DTU, const double2* DTD,
                           const double2* DTDU, const double2* X01, const double2* X10, const double2* X00,
                           const double2* f, const double* epsh, const double* E0p, double b, double s,
                           const double2* g1, double2* T, double* H, double* GV, double* part);
__global__ void k_gather_fock(int cls, DevList Lx, DevList Lsrc, DevDas das, DevSpace sp, const int64_t* binom,
                              const double2* Dsrc, const double2* T, double2* Gf);
__global__ void k_gather_d1(int cls, DevList Lx, DevList Ltab, DevDas das, DevSpace sp, const int64_t* binom,
                            const double2* T, int nrow, const double2* f, double2* GD);
__global__ void k_gather_d2(int cls, DevList Lx, DevList Ltab, DevDas das, DevSpace sp, const int64_t* binom,
                            const double2* T, int nrow, const double2* X, double2* GD);
__global__ void k_dscatter(int fam, DevList Ls, DevList Pl, DevDas das, const int64_t* binom, const double2* GD,
                           double2* Gc);
__global__ void k_sum2(const double* H, const double* GV, int64_t n, double* scal);
__global__ void k_e0grad(const double2* g1, const double* scal, DevSpace sp, double2* Gf);
__global__ void k_nd(DevSpace sp, const double* Nx, const double* Nt, double* Nd);
__global__ void k_cbar(int64_t np, const double2* Gc, const double* c22, const double2* c, const double2* sigma,
                       const double* scal, const double* E0p, const double2* g1, double2* out);
__global__ void k_hbar(DevSpace sp, const double2* Gf, const double* Nd, double2* gh);

__global__ void k_dgemm(int64_t M, int64_t N, int64_t K, const double* A, int64_t sam, int64_t sak, const double* B,
                        int64_t sbk, int64_t sbn, double* C, int64_t ldc, int beta, int64_t kseg, int64_t czs);
__global__ void k_dacc(const double* part, int nseg, int64_t ps, int64_t count, double* out);
__global__ void k_hocc(const double* H, DevList Ls, int na, double* Hocc, const int32_t* perm,
                       int64_t ld);
__global__ void k_tmarg(const double* in, int64_t nb, int64_t nt, int w, int arity, int ns, double sign, int acc,
                        double* out, int64_t ob, int64_t os, int64_t oc);
__global__ void k_pairplace(const double* in, int ns, double* out, int64_t ldo);
__global__ void k_midsum(const double* in, int64_t np, int w, double* out);
__global__ void k_gint(int mode, DevSpace sp, const double2* Gam, int64_t rows, int cols, int ld, double2* Gt,
                       int64_t npair);
__global__ void k_tshift(DevList Lx, DevList Ltab, DevDas das, const int64_t* binom, const double2* T, int row0,
                         int pairs_mode, double2* Tsh);
__global__ void k_class22_rows(DevList Ls, DevSpace sp, const double2* c, const double* g2, const double* epsh,
                               const double* G, const double* E0p, double b, double s, const double2* g1, double* hsum,
                               double* Hocc, double* P22);
__global__ void k_g22coef(const double2* g, const double* P22, int64_t n, double2* out);
__global__ void k_ntt(DevList Ls, const double* hA, int na, double* Ntt);
__global__ void k_gg(DevSpace sp, const double* Nd, const double* Ntt, const double* Ge, const double* Gea, double* GG);
__global__ void k_symm(const double2* Gt, int64_t npair, double2* Gh);
__global__ void k_bcoef(DevSpace sp, const double2* Bc, const double2* Bx, int Lc, int Lx, const double* wt,
                        const double* dg, const double2* Cs, const double* GG, const double2* Gf, const double2* ftr,
                        double2* GB);
__global__ void k_ftr(DevSpace sp, const double2* Bc, const double2* Bx, int Lc, const double2* Gf, double2* ftr);
__global__ void k_gw(DevSpace sp, const double2* Bc, const double2* Bx, int Lc, const double2* Bo, const double2* Cs,
                     const double* GG, const double2* Gf, const double* dg, double* gw);
__global__ void k_bproj(int n, int Lc, int Lx, const double2* GB, double2* gBc, double2* gBx);
__global__ void k_x00e0(const double2* g1, const double2* g2, const double* scal, int ntp, double2* GX00);
__global__ void k_dlambda(const double* gw, const double* wx, int Lc, int Lx, double* out);

}  // namespace e2
