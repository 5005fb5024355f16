// sm_103a kernels of the Epstein-Nesbet second-order energy (Sec. 2.3-2.6).
//
// Notation: i, j correlated core spinors; t, u, v, w active; a, b correlated
// virtual; A an active string (bitset over active-local indices).
//   <pq||rs> = (pr|qs) - (ps|qr),  (pq|rs) = sum_L wt_L B^L_pq B^L_rs
//   G_pq = <pq||pq>,  eps^_p = h_pp + sum_{k in core} G_pk,
//   f_pq = h_pq + sum_{k in core} <pk||qk>   (h^FC of Sec. 2 over the whole core)
//   H_KK = E_O + e_A + chi(e) + sum_{s in S} U[s,A] - sum_{i in I} U[i,A]
// Every class's coupling V_K = <K|H|Psi> is, up to a sign per external
// tuple that cancels in |V_K|^2, a contraction sum_x W[e,x] D^x_A of
// integrals with active coupling tensors D^x_A = <A|x|Psi>.
#include <cuda_runtime.h>

#include "e2_common.cuh"
#include "e2_kernels.cuh"
#include "e2_device.cuh"

namespace e2 {

// ------------------------------------------------------------------ setup

__global__ void k_binom(int64_t* tab) {
  for (int idx = threadIdx.x; idx < kBinomN * kBinomN; idx += blockDim.x) {
    int n = idx / kBinomN, k = idx % kBinomN;
    // C(n,k) by the multiplicative formula with exact integer steps
    int64_t r = (k > n) ? 0 : 1;
    if (k <= n) {
      int kk = k < n - k ? k : n - k;
      for (int j = 1; j <= kk; ++j) r = r * (n - kk + j) / j;
    }
    tab[idx] = r;
  }
}

// Bo[L][p][y] = B^L_py for y < n_occ (core + active), all factor sets
// concatenated; wt[L] = 1 (Coulomb) or lambda * w_x (Gaunt / Breit).
__global__ void k_extract(const double2* __restrict__ Bc, const double2* __restrict__ Bx, const double* __restrict__ wx,
                          double lambda, int Lc, int Lx, int n, int nocc, double2* __restrict__ Bo,
                          double* __restrict__ wt, double* __restrict__ dg) {
  int64_t total = (int64_t)(Lc + Lx) * n * nocc;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    int y = (int)(idx % nocc);
    int64_t r = idx / nocc;
    int p = (int)(r % n);
    int L = (int)(r / n);
    const double2* src = (L < Lc) ? Bc + (int64_t)L * n * n : Bx + (int64_t)(L - Lc) * n * n;
    Bo[idx] = src[(int64_t)p * n + y];
  }
  int64_t tot2 = (int64_t)(Lc + Lx) * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot2; idx += (int64_t)gridDim.x * blockDim.x) {
    int p = (int)(idx % n);
    int L = (int)(idx / n);
    const double2* src = (L < Lc) ? Bc + (int64_t)L * n * n : Bx + (int64_t)(L - Lc) * n * n;
    dg[idx] = src[(int64_t)p * n + p].x;
    if (p == 0) wt[L] = (L < Lc) ? 1.0 : lambda * wx[L - Lc];
  }
}

// G_pq = (pp|qq) - (pq|qp) = sum_L wt_L (B_pp B_qq - |B_pq|^2)  (B Hermitian)
__global__ void k_G(const double2* __restrict__ Bc, const double2* __restrict__ Bx, const double* __restrict__ wt,
                    const double* __restrict__ dg, int Lc, int Lx, int n, double* __restrict__ G) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  int p = (int)(idx / n), q = (int)(idx % n);
  double acc = 0.0;
  for (int L = 0; L < Lc + Lx; ++L) {
    const double2* src = (L < Lc) ? Bc + (int64_t)L * n * n : Bx + (int64_t)(L - Lc) * n * n;
    double2 b = src[idx];
    double v = dg[(int64_t)L * n + p] * dg[(int64_t)L * n + q] - (b.x * b.x + b.y * b.y);
    acc = fma(wt[L], v, acc);
  }
  G[idx] = (p == q) ? 0.0 : acc;
}

// f[p][y] = h_py + sum_L wt_L (B_py sum_k B_kk - sum_k B_pk B_ky), y < n_occ
__global__ void k_fock(const double2* __restrict__ h, const double2* __restrict__ Bo, const double* __restrict__ wt,
                       const double* __restrict__ dg, int L, int n, int nocc, int ncore, double2* __restrict__ f) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * nocc) return;
  int p = (int)(idx / nocc), y = (int)(idx % nocc);
  double2 acc = h[(int64_t)p * n + y];
  for (int l = 0; l < L; ++l) {
    const double2* B = Bo + (int64_t)l * n * nocc;
    double trc = 0.0;
    for (int k = 0; k < ncore; ++k) trc += dg[(int64_t)l * n + k];
    double2 bpy = B[(int64_t)p * nocc + y];
    double2 s = make_double2(bpy.x * trc, bpy.y * trc);
    for (int k = 0; k < ncore; ++k) {
      double2 m = cmul(B[(int64_t)p * nocc + k], B[(int64_t)k * nocc + y]);
      s.x -= m.x;
      s.y -= m.y;
    }
    acc.x = fma(wt[l], s.x, acc.x);
    acc.y = fma(wt[l], s.y, acc.y);
  }
  f[idx] = acc;
}

// eps^_p = h_pp + sum_{k<ncore} G_pk ; E_O = sum_k h_kk + 1/2 sum_kl G_kl
__global__ void k_scalars(const double2* __restrict__ h, const double* __restrict__ G, int n, int ncore,
                          double* __restrict__ epsh, double* __restrict__ EO) {
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    double s = h[(int64_t)p * n + p].x;
    for (int k = 0; k < ncore; ++k) s += G[(int64_t)p * n + k];
    epsh[p] = s;
  }
  __shared__ double red[256];
  double part = 0.0;
  for (int k = threadIdx.x; k < ncore; k += blockDim.x) {
    double s = h[(int64_t)k * n + k].x;
    for (int l = 0; l < ncore; ++l) s += 0.5 * G[(int64_t)k * n + l];
    part += s;
  }
  red[threadIdx.x] = part;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *EO = red[0];
}

// String list: unrank every entry (pattern block, then mixed radix over
// subspaces with subspace 1 fastest, colex inside each subspace).
__global__ void k_unrank(DevList Ls, DevDas das, const int64_t* __restrict__ binom) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= Ls.n) return;
  int k = 0;
  while (k + 1 < Ls.npat && Ls.patoff[k + 1] <= g) ++k;
  int64_t r = g - Ls.patoff[k];
  uint64_t A = 0;
  for (int s = 0; s < das.n_das; ++s) {
    int occ = Ls.patocc[k * E2_MAX_DAS + s];
    int64_t cnt = binom[das.size[s] * kBinomN + occ];
    int64_t rk = r % cnt;
    r /= cnt;
    A |= colex_unrank(rk, occ, das.size[s], binom) << das.off[s];
  }
  Ls.str[g] = A;
}

// e_A = sum_{t in A} eps^_t + 1/2 sum_{t != u in A} G_tu
__global__ void k_eA(DevList Ls, const double* __restrict__ epsh, const double* __restrict__ G, int n, int a0) {
  int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= Ls.n) return;
  uint64_t A = Ls.str[g];
  double e = 0.0;
  for (uint64_t x = A; x; x &= x - 1) {
    int t = __ffsll((long long)x) - 1;
    e += epsh[a0 + t];
    for (uint64_t y = x & (x - 1); y; y &= y - 1) {
      int u = __ffsll((long long)y) - 1;
      e += G[(int64_t)(a0 + t) * n + a0 + u];
    }
  }
  Ls.eA[g] = e;
}

// U[x][A] = sum_{t in A} G_{X(x), t}; X = correlated core then correlated virtual.
__global__ void k_U(DevList Ls, DevSpace sp, const double* __restrict__ G) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = (int64_t)(sp.nx + 1) * Ls.n;
  if (idx >= total) return;
  int x = (int)(idx / Ls.n);
  int64_t g = idx % Ls.n;
  double s = 0.0;
  if (x < sp.nx) {
    int p = (x < sp.ncc) ? sp.cc[x] : sp.vc[x - sp.ncc];
    for (uint64_t A = Ls.str[g]; A; A &= A - 1) s += G[(int64_t)p * sp.n + sp.a0 + __ffsll((long long)A) - 1];
  }
  Ls.U[idx] = s;
}

// ------------------------------------------------------------------ integrals

// B^L_pq through the compact factors: q < n_occ read directly, else
// p < n_occ and B_pq = conj(B_qp) (Hermitian factors).
__device__ __forceinline__ double2 Bget(const double2* __restrict__ Bo, int n, int nocc, int p, int q) {
  if (q < nocc) return Bo[(int64_t)p * nocc + q];
  return cconj(Bo[(int64_t)q * nocc + p]);
}

// <pq||rs> = sum_L wt_L (B_pr B_qs - B_ps B_qr)
__device__ double2 asym(const double2* __restrict__ Bo, const double* __restrict__ wt, int L, int n, int nocc, int p,
                        int q, int r, int s) {
  double2 acc = make_double2(0.0, 0.0);
  const int64_t stride = (int64_t)n * nocc;
  for (int l = 0; l < L; ++l) {
    const double2* B = Bo + l * stride;
    double2 x = cmul(Bget(B, n, nocc, p, r), Bget(B, n, nocc, q, s));
    double2 y = cmul(Bget(B, n, nocc, p, s), Bget(B, n, nocc, q, r));
    acc.x = fma(wt[l], x.x - y.x, acc.x);
    acc.y = fma(wt[l], x.y - y.y, acc.y);
  }
  return acc;
}

__global__ void k_integrals(int mode, DevSpace sp, const double2* __restrict__ Bo, const double* __restrict__ wt, int L,
                            const double2* __restrict__ f, int64_t rows, int cols, int ld, void* out) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= rows * (int64_t)ld) return;
  int64_t row = idx / ld;
  int col = (int)(idx % ld);
  double2 v = make_double2(0.0, 0.0);
  if (col < cols) {
    int p, q, r, s;
    if (int_indices(mode, sp, row, col, p, q, r, s)) v = f[(int64_t)p * sp.n_occ + q];
    else v = asym(Bo, wt, L, sp.n, sp.n_occ, p, q, r, s);
  }
  if (mode == INT_G22) ((double*)out)[idx] = v.x * v.x + v.y * v.y;
  else ((double2*)out)[idx] = v;
}

// Factor columns of the (virtual, active) pairs, nva = nvc * na:
//   Yw[(a*na + t)*Lt + L] = wt_L B^L_{a t}   (row-major in the pair)
//   Zt[L*nva + a*na + t] = B^L_{a t}         (row-major in L)
__global__ void k_vafactors(DevSpace sp, const double2* __restrict__ Bo, const double* __restrict__ wt, int Lt,
                            double2* __restrict__ Yw, double2* __restrict__ Zt) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int na = sp.n_act;
  const int64_t nva = (int64_t)sp.nvc * na;
  if (idx >= nva * Lt) return;
  const int L = (int)(idx / nva);
  const int64_t at = idx % nva;
  const int a = (int)(at / na), t = (int)(at % na);
  const double2 b = Bo[((int64_t)L * sp.n + sp.vc[a]) * sp.n_occ + sp.a0 + t];
  Zt[idx] = b;
  Yw[at * Lt + L] = make_double2(wt[L] * b.x, wt[L] * b.y);
}

// Factor columns of (virtual, core) pairs and of active pairs:
//   Ywc[(a*ncc + i)*Lt + L] = wt_L B^L_{a i},  Zaa[L*na*na + u*na + w] = B^L_{u w}
__global__ void k_xfactors(DevSpace sp, const double2* __restrict__ Bo, const double* __restrict__ wt, int Lt,
                           double2* __restrict__ Ywc, double2* __restrict__ Zaa) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int na = sp.n_act;
  const int64_t nvc = (int64_t)sp.nvc * sp.ncc * Lt, naa = (int64_t)na * na * Lt;
  if (idx < nvc) {
    const int L = (int)(idx % Lt);
    const int64_t ai = idx / Lt;
    const int a = (int)(ai / sp.ncc), i = (int)(ai % sp.ncc);
    const double2 b = Bo[((int64_t)L * sp.n + sp.vc[a]) * sp.n_occ + sp.cc[i]];
    Ywc[idx] = make_double2(wt[L] * b.x, wt[L] * b.y);
  } else if (idx < nvc + naa) {
    const int64_t r = idx - nvc;
    const int L = (int)(r / (na * na));
    const int uw = (int)(r % (na * na));
    Zaa[r] = Bo[((int64_t)L * sp.n + sp.a0 + uw / na) * sp.n_occ + sp.a0 + uw % na];
  }
}

// <ab||it> = (ai|bt) - (at|bi) from X[(a*ncc + i)*ldx + b*na + t] = (ai|bt):
// rows (i, a<b) = i * npair_v + pair(a,b), columns t padded to Kp with zeros
__global__ void k_w12(DevSpace sp, const double2* __restrict__ X, int64_t ldx, int64_t M, int Kp,
                      double2* __restrict__ W) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= M * Kp) return;
  const int64_t row = idx / Kp;
  const int t = (int)(idx % Kp), na = sp.n_act;
  double2 v = make_double2(0.0, 0.0);
  if (t < na) {
    const int64_t nvp = pairs(sp.nvc);
    const int i = (int)(row / nvp);
    int a, b;
    pair_decode(row % nvp, a, b);
    const double2 x1 = X[((int64_t)a * sp.ncc + i) * ldx + (int64_t)b * na + t];
    const double2 x2 = X[((int64_t)b * sp.ncc + i) * ldx + (int64_t)a * na + t];
    v = make_double2(x1.x - x2.x, x1.y - x2.y);
  }
  W[idx] = v;
}

// <au||vw> = (av|uw) - (aw|uv) from X[(a*na + v)*na*na + u*na + w] = (av|uw):
// rows a, columns u * ntp + pair(v,w)
__global__ void k_x01(DevSpace sp, const double2* __restrict__ X, double2* __restrict__ X01) {
  const int na = sp.n_act, ntp = (int)pairs(na);
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)sp.nvc * na * ntp) return;
  const int a = (int)(idx / ((int64_t)na * ntp));
  const int col = (int)(idx % ((int64_t)na * ntp));
  const int u = col / ntp;
  int v, w;
  pair_decode(col % ntp, v, w);
  const int64_t n2 = (int64_t)na * na;
  const double2 x1 = X[((int64_t)a * na + v) * n2 + u * na + w];
  const double2 x2 = X[((int64_t)a * na + w) * n2 + u * na + v];
  X01[idx] = make_double2(x1.x - x2.x, x1.y - x2.y);
}

// <ab||tu> = (at|bu) - (au|bt) for the rows (a<b) with b0 <= b < b1 (a
// contiguous run of rows in pair order), columns (t<u) padded to Kp with zeros,
// from a stripe X[(b*na + u - b0*na)*ldx + a*na + t] = (at|bu), a < b.
__global__ void k_w02(DevSpace sp, const double2* __restrict__ X, int64_t ldx, int b0, int b1, int Kp,
                      double2* __restrict__ W) {
  const int64_t r0 = pairs(b0), nrow = pairs(b1) - r0;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nrow * Kp) return;
  const int64_t row = r0 + idx / Kp;
  const int col = (int)(idx % Kp);
  const int na = sp.n_act;
  double2 v = make_double2(0.0, 0.0);
  if (col < (int)pairs(na)) {
    int a, b, t, u;
    pair_decode(row, a, b);
    pair_decode(col, t, u);
    const double2* Xb = X + (int64_t)(b - b0) * na * ldx;
    const double2 x1 = Xb[(int64_t)u * ldx + (int64_t)a * na + t];
    const double2 x2 = Xb[(int64_t)t * ldx + (int64_t)a * na + u];
    v = make_double2(x1.x - x2.x, x1.y - x2.y);
  }
  W[row * Kp + col] = v;
}

// Row descriptors of the dense classes: U rows of particles / holes and
// chi(e) = -sum_I eps^_i + [h=2] G_ij + sum_S eps^_s + [p=2] G_ab - sum_{IxS} G.
// Two holes in one core subspace, or two particles in one virtual subspace,
// whose limit is one (correlated-space indices; -1 = absent).
__device__ __forceinline__ bool row_excluded(const DevSpace& sp, int i0, int i1, int a0, int a1) {
  if (i0 >= 0 && i1 >= 0 && sp.xc[i0] >= 0 && sp.xc[i0] == sp.xc[i1]) return true;
  if (a0 >= 0 && a1 >= 0 && sp.xv[a0] >= 0 && sp.xv[a0] == sp.xv[a1]) return true;
  return false;
}

__device__ RowInfo row_info(int cls, const DevSpace& sp, const double* __restrict__ epsh,
                            const double* __restrict__ G, int64_t row) {
  const int nvp = (int)pairs(sp.nvc);
  int I[2] = {-1, -1}, S[2] = {-1, -1}, x, y;
  switch (cls) {
    case 2: pair_decode(row, x, y); S[0] = x; S[1] = y; break;                                     // (0,2)
    case 5: I[0] = (int)(row / nvp); pair_decode(row % nvp, x, y); S[0] = x; S[1] = y; break;      // (1,2)
    case 7: S[0] = (int)(row % sp.nvc); pair_decode(row / sp.nvc, x, y); I[0] = x; I[1] = y; break;  // (2,1)
    case 4: I[0] = (int)(row / sp.nvc); S[0] = (int)(row % sp.nvc); break;                           // (1,1)
    case 6: pair_decode(row, x, y); I[0] = x; I[1] = y; break;                                     // (2,0)
    case 1: S[0] = (int)row; break;                                                                 // (0,1)
    case 3: I[0] = (int)row; break;                                                                 // (1,0)
    case 8: {                                                                                       // (2,2)
      const int64_t nv2 = nvp;
      pair_decode(row / nv2, x, y); I[0] = x; I[1] = y;
      pair_decode(row % nv2, x, y); S[0] = x; S[1] = y;
    } break;
    default: break;                                                                                 // (0,0)
  }
  double chi = 0.0;
  int gi[2], gs[2];
  for (int k = 0; k < 2; ++k) {
    gi[k] = I[k] >= 0 ? sp.cc[I[k]] : -1;
    gs[k] = S[k] >= 0 ? sp.vc[S[k]] : -1;
  }
  for (int k = 0; k < 2; ++k) {
    if (gi[k] >= 0) chi -= epsh[gi[k]];
    if (gs[k] >= 0) chi += epsh[gs[k]];
  }
  if (gi[1] >= 0) chi += G[(int64_t)gi[0] * sp.n + gi[1]];
  if (gs[1] >= 0) chi += G[(int64_t)gs[0] * sp.n + gs[1]];
  for (int k = 0; k < 2; ++k)
    for (int l = 0; l < 2; ++l)
      if (gi[k] >= 0 && gs[l] >= 0) chi -= G[(int64_t)gi[k] * sp.n + gs[l]];
  RowInfo ri;
  ri.s1 = S[0] >= 0 ? sp.ncc + S[0] : sp.nx;
  ri.s2 = S[1] >= 0 ? sp.ncc + S[1] : sp.nx;
  ri.i1 = I[0] >= 0 ? I[0] : sp.nx;
  ri.i2 = I[1] >= 0 ? I[1] : sp.nx;
  ri.chi = row_excluded(sp, I[0], I[1], S[0], S[1]) ? kExcludedChi : chi;
  return ri;
}

// Zero the W rows of excluded external rows (their V is then 0).
__global__ void k_mask_rows(double2* __restrict__ W, int64_t M, int Kp, const RowInfo* __restrict__ rows) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= M * Kp) return;
  if (rows[idx / Kp].chi == kExcludedChi) W[idx] = make_double2(0.0, 0.0);
}

// Zero the class-(2,2) entries [(i<j)][(a<b)] of excluded rows: |<ab||ij>|^2
// (cplx = 0) or <ab||ij> (cplx = 1).
__global__ void k_mask22(void* __restrict__ g, int64_t ncp, int64_t nvp, DevSpace sp, int cplx) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= ncp * nvp) return;
  int i, j, a, b;
  pair_decode(idx / nvp, i, j);
  pair_decode(idx % nvp, a, b);
  if (!row_excluded(sp, i, j, a, b)) return;
  if (cplx) ((double2*)g)[idx] = make_double2(0.0, 0.0);
  else ((double*)g)[idx] = 0.0;
}

__global__ void k_rows(int cls, DevSpace sp, const double* __restrict__ epsh, const double* __restrict__ G, int64_t M,
                       RowInfo* __restrict__ out) {
  int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= M) return;
  out[row] = row_info(cls, sp, epsh, G, row);
}

// Histogram of |D|, D = E0' - chi_e - e_A - U[s1,A] - U[s2,A] + U[i1,A] + U[i2,A],
// over the couplings of one class (intruder diagnostics, Sec. 2.6): bin 0
// |D| < 1e-12, bin k = 1..DHIST-2: 10^(k-13) <= |D| < 10^(k-12), the last bin
// the rest (and NaN).  Grid: x = external rows, y = chunks of 4096 strings.
constexpr int DHIST = 18;
__global__ void __launch_bounds__(256) k_dhist(int cls, DevSpace sp, DevList L, const double* __restrict__ epsh,
                                               const double* __restrict__ G, const double* __restrict__ E0p,
                                               unsigned long long* __restrict__ hist) {
  __shared__ unsigned sh[DHIST];
  __shared__ RowInfo sri;
  if (threadIdx.x < DHIST) sh[threadIdx.x] = 0;
  if (threadIdx.x == 0) sri = row_info(cls, sp, epsh, G, blockIdx.x);
  __syncthreads();
  const RowInfo ri = sri;
  if (ri.chi == kExcludedChi) return;  // not in Q (external subspace limits)
  const double base = *E0p - ri.chi;
  const double* U1 = L.U + (int64_t)ri.s1 * L.n;
  const double* U2 = L.U + (int64_t)ri.s2 * L.n;
  const double* U3 = L.U + (int64_t)ri.i1 * L.n;
  const double* U4 = L.U + (int64_t)ri.i2 * L.n;
  const int64_t a0 = (int64_t)blockIdx.y * 4096, a1 = min(L.n, a0 + 4096);
  for (int64_t A = a0 + threadIdx.x; A < a1; A += blockDim.x) {
    const double D = fabs(base - L.eA[A] - U1[A] - U2[A] + U3[A] + U4[A]);
    int k;
    if (D < 1e-12) {
      k = 0;
    } else {
      k = DHIST - 1;
      double edge = 1e-11;
      for (int q = 1; q < DHIST - 1; ++q, edge *= 10.0)
        if (D < edge) {
          k = q;
          break;
        }
    }
    atomicAdd(&sh[k], 1u);
  }
  __syncthreads();
  if (threadIdx.x < DHIST && sh[threadIdx.x]) atomicAdd(hist + threadIdx.x, (unsigned long long)sh[threadIdx.x]);
}

// ------------------------------------------------------------------ D tables

// D[x][A] = <A| x |Psi_m> for one family over list Ls; c in P-address order.
__global__ void k_dtable(int fam, DevList Ls, DevList Pl, DevDas das, const int64_t* __restrict__ binom,
                         const double2* __restrict__ c, int Kp, double2* __restrict__ D) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)Kp * Ls.n) return;
  int xr = (int)(idx / Ls.n);
  int64_t g = idx % Ls.n;
  const uint64_t A = Ls.str[g];
  const int na = das.n_act;
  uint64_t Lb = 0;
  int sign = 0;  // 0: zero entry
  switch (fam) {
    case FAM_T: {  // a_t on L = A + t
      if (xr < na && !((A >> xr) & 1)) {
        Lb = A | (1ull << xr);
        sign = (popc_below(A, xr) & 1) ? -1 : 1;
      }
    } break;
    case FAM_TD: {  // a+_t on L = A - t
      if (xr < na && ((A >> xr) & 1)) {
        Lb = A & ~(1ull << xr);
        sign = (popc_below(A, xr) & 1) ? -1 : 1;
      }
    } break;
    case FAM_TU: {  // a_u a_t on L = A + t + u
      if (xr < (int)pairs(na)) {
        int t, u;
        pair_decode(xr, t, u);
        if (!((A >> t) & 1) && !((A >> u) & 1)) {
          Lb = A | (1ull << t) | (1ull << u);
          int par = popc_below(Lb, t) + popc_below(Lb & ~(1ull << t), u);
          sign = (par & 1) ? -1 : 1;
        }
      }
    } break;
    case FAM_TDUD: {  // a+_t a+_u on B = A - t - u
      if (xr < (int)pairs(na)) {
        int t, u;
        pair_decode(xr, t, u);
        if (((A >> t) & 1) && ((A >> u) & 1)) {
          Lb = A & ~(1ull << t) & ~(1ull << u);
          int par = popc_below(Lb, u) + popc_below(Lb, t);
          sign = (par & 1) ? -1 : 1;
        }
      }
    } break;
    case FAM_TDU: {  // row 0: c_A ; row 1+t*na+u: a+_t a_u on L = A - t + u
      if (xr == 0) {
        Lb = A;
        sign = 1;
      } else if (xr <= na * na) {
        int t = (xr - 1) / na, u = (xr - 1) % na;
        if (((A >> t) & 1) && (u == t || !((A >> u) & 1))) {
          Lb = (A & ~(1ull << t)) | (1ull << u);
          int par = popc_below(Lb, u) + popc_below(A, t);
          sign = (par & 1) ? -1 : 1;
        }
      }
    } break;
  }
  double2 v = make_double2(0.0, 0.0);
  if (sign != 0) {
    int64_t ad = list_addr(Pl, das, binom, Lb);
    if (ad >= 0) {
      v = c[ad];
      if (sign < 0) v = make_double2(-v.x, -v.y);
    }
  }
  D[idx] = v;
}

// ------------------------------------------------------------------ E0

// out[x][y] = sum_A conj(Da[x][A]) Db[y][A]  (one block per (x, y))
__global__ void k_gram(const double2* __restrict__ Da, const double2* __restrict__ Db, int64_t n, int ny,
                       double2* __restrict__ out) {
  __shared__ double sh[32];
  const int x = blockIdx.x / ny, y = blockIdx.x % ny;
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t g = threadIdx.x; g < n; g += blockDim.x) acc = cfma(cconj(Da[(int64_t)x * n + g]), Db[(int64_t)y * n + g], acc);
  double re = block_sum(acc.x, sh);
  double im = block_sum(acc.y, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = make_double2(re, im);
}

// E0' = (sum_tu f_tu gamma_tu + sum_{x,y} <x||y> Gamma_xy) / <c|c>,
// gamma_tu = <Psi|a+_t a_u|Psi>, Gamma_{(tu),(vw)} = <Psi|a+_t a+_u a_w a_v|Psi>.
__global__ void k_e0(const double2* __restrict__ g1 /*[1+na*na] row 0 = <c|c>*/, const double2* __restrict__ g2,
                     const double2* __restrict__ f, const double2* __restrict__ X00, DevSpace sp, int ntp,
                     const double* __restrict__ EO, double* __restrict__ E0p, double* __restrict__ E0) {
  __shared__ double sh[32];
  const int na = sp.n_act;
  double acc = 0.0;
  for (int k = threadIdx.x; k < na * na; k += blockDim.x) {
    int t = k / na, u = k % na;
    double2 fv = f[(int64_t)(sp.a0 + t) * sp.n_occ + sp.a0 + u];
    double2 gv = g1[1 + k];
    acc += fv.x * gv.x - fv.y * gv.y;
  }
  for (int k = threadIdx.x; k < ntp * ntp; k += blockDim.x) {
    double2 xv = X00[k], gv = g2[k];
    acc += xv.x * gv.x - xv.y * gv.y;
  }
  double tot = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    double e = tot / g1[0].x;
    *E0p = e;
    *E0 = e + *EO;
  }
}

// ------------------------------------------------------------------ dense classes

// V[e,A] = sum_x W[e,x] D[x,A] on the FP64 tensor pipe (mma.sync m16n8k8
// f64), with the Epstein-Nesbet denominator and |V|^2/D reduced in the
// epilogue; V is never stored.  Complex products take three real products
// (Gauss): T1 = Wr Dr, T2 = Wi Di, T3 = (Wr + Wi)(Dr + Di), Re V = T1 - T2,
// Im V = T3 - T1 - T2; the sums are formed once per tile in shared memory.
// CTA tile 64x64, 8 warps of 32x16, K steps of 8 with the next step's tile
// prefetched into registers; one partial per CTA.
constexpr int GBM = 64, GBN = 64, GBK = 8;

__device__ __forceinline__ void class_tile(const double2* __restrict__ W, const double2* __restrict__ D, int64_t M,
                                           int64_t N, int Kp, const RowInfo* __restrict__ rows,
                                           const double* __restrict__ U, const double* __restrict__ eA,
                                           const double* __restrict__ E0p, double b, double* __restrict__ partial_slot,
                                           const AdjOut& adj, int64_t tile_m, int64_t tile_n, int64_t n_tile_n,
                                           const ColTiles& ctl, unsigned long long* dmin) {
  __shared__ double sWr[GBM][GBK + 1], sWi[GBM][GBK + 1], sWs[GBM][GBK + 1];
  __shared__ double sDr[GBK][GBN + 1], sDi[GBK][GBN + 1], sDs[GBK][GBN + 1];
  __shared__ double sh[32];
  __shared__ int32_t sCol[GBN];   // list index of each tile column (-1: none)
  __shared__ int32_t sK[512];     // compacted D rows of this tile (staged in 512-row windows)
  // tile (tile_m, tile_n): rows from m_base + 64 tile_m, columns from 64 tile_n
  // (through perm for a compacted class)
  const int64_t m0 = adj.m_base + tile_m * GBM, n0 = tile_n * GBN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool sparse = ctl.perm != nullptr;
  int koff = 0, klen = Kp;
  if (sparse) {
    const int4 td = ctl.tdesc[tile_n];
    koff = td.x;
    klen = td.y;
    D = ctl.Dc + (int64_t)koff * GBN;  // compacted rows of this tile, 64 wide
  }
  if (tid < GBN) sCol[tid] = sparse ? ctl.perm[n0 + tid] : (n0 + tid < N ? (int32_t)(n0 + tid) : -1);
  const int64_t ldd = sparse ? GBN : N;    // row stride of the B operand
  const int64_t dcol0 = sparse ? 0 : n0;   // its first column
  const int g = lane >> 2, tq = lane & 3;
  const int wm = warp >> 2, wn = warp & 3;  // warp tile: rows wm*32.., cols wn*16..
  double t1[2][2][4], t2[2][2][4], t3[2][2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e) t1[a][c][e] = t2[a][c][e] = t3[a][c][e] = 0.0;

  // per thread: two W elements (rows r, r+32 of the 64x8 tile) and two D
  // elements (k rows kr, kr+4 of the 8x64 tile)
  const int wr_ = tid >> 3, wk = tid & 7, dk = tid >> 6, dc = tid & 63;
  const double2 zero = make_double2(0.0, 0.0);
  // W column of compacted row k: staged window [kw0, kw0 + 512) of klist
  int kw0 = 0;
  auto stage = [&](int k0) {
    kw0 = k0;
    for (int i = tid; i < 512 && k0 + i < klen; i += blockDim.x) sK[i] = ctl.klist[koff + k0 + i];
  };
  if (sparse) stage(0);
  __syncthreads();
  auto wcol = [&](int k) { return sparse ? sK[k - kw0] : k; };
  const bool colok = dcol0 + dc < N || sparse;
  // rows past klen (a k = 4 tail of a compacted tile) read zero
  auto ldW = [&](int k0, int q) {
    const int64_t gr = m0 + wr_ + 32 * q;
    return (gr < M && k0 + wk < klen) ? W[gr * Kp + wcol(k0 + wk)] : zero;
  };
  auto ldD = [&](int k0, int q) {
    return (colok && k0 + dk + 4 * q < klen) ? D[(int64_t)(k0 + dk + 4 * q) * ldd + dcol0 + dc] : zero;
  };
  double2 pw0 = ldW(0, 0), pw1 = ldW(0, 1), pd0 = ldD(0, 0), pd1 = ldD(0, 1);

  for (int k0 = 0; k0 < klen; k0 += GBK) {
    sWr[wr_][wk] = pw0.x; sWi[wr_][wk] = pw0.y; sWs[wr_][wk] = pw0.x + pw0.y;
    sWr[wr_ + 32][wk] = pw1.x; sWi[wr_ + 32][wk] = pw1.y; sWs[wr_ + 32][wk] = pw1.x + pw1.y;
    sDr[dk][dc] = pd0.x; sDi[dk][dc] = pd0.y; sDs[dk][dc] = pd0.x + pd0.y;
    sDr[dk + 4][dc] = pd1.x; sDi[dk + 4][dc] = pd1.y; sDs[dk + 4][dc] = pd1.x + pd1.y;
    __syncthreads();
    if (k0 + GBK < klen) {  // prefetch the next K step while the tensor pipe works
      if (sparse && k0 + GBK - kw0 >= 512) {  // next klist window (all threads are past their reads)
        __syncthreads();
        stage(k0 + GBK);
        __syncthreads();
      }
      pw0 = ldW(k0 + GBK, 0);
      pw1 = ldW(k0 + GBK, 1);
      pd0 = ldD(k0 + GBK, 0);
      pd1 = ldD(k0 + GBK, 1);
    }
    double br[2][2], bi[2][2], bs[2][2];
#pragma unroll
    for (int ni = 0; ni < 2; ++ni) {
      const int cb = wn * 16 + ni * 8 + g;
      br[ni][0] = sDr[tq][cb]; br[ni][1] = sDr[tq + 4][cb];
      bi[ni][0] = sDi[tq][cb]; bi[ni][1] = sDi[tq + 4][cb];
      bs[ni][0] = sDs[tq][cb]; bs[ni][1] = sDs[tq + 4][cb];
    }
    if (k0 + GBK <= klen) {
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r0 = wm * 32 + mi * 16 + g;
        double a[4];
        a[0] = sWr[r0][tq]; a[1] = sWr[r0 + 8][tq]; a[2] = sWr[r0][tq + 4]; a[3] = sWr[r0 + 8][tq + 4];
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) mma_f64(t1[mi][ni], a, br[ni]);
        a[0] = sWi[r0][tq]; a[1] = sWi[r0 + 8][tq]; a[2] = sWi[r0][tq + 4]; a[3] = sWi[r0 + 8][tq + 4];
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) mma_f64(t2[mi][ni], a, bi[ni]);
        a[0] = sWs[r0][tq]; a[1] = sWs[r0 + 8][tq]; a[2] = sWs[r0][tq + 4]; a[3] = sWs[r0 + 8][tq + 4];
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) mma_f64(t3[mi][ni], a, bs[ni]);
      }
    } else {  // k = 4 tail: the first four staged rows (m16n8k4 fragments)
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r0 = wm * 32 + mi * 16 + g;
        double a[2];
        a[0] = sWr[r0][tq]; a[1] = sWr[r0 + 8][tq];
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) mma_f64_k4(t1[mi][ni], a, br[ni][0]);
        a[0] = sWi[r0][tq]; a[1] = sWi[r0 + 8][tq];
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) mma_f64_k4(t2[mi][ni], a, bi[ni][0]);
        a[0] = sWs[r0][tq]; a[1] = sWs[r0 + 8][tq];
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) mma_f64_k4(t3[mi][ni], a, bs[ni][0]);
      }
    }
    __syncthreads();
  }

  // epilogue: D_K = E0' - chi(e) - e_A - U[s1,A] - U[s2,A] + U[i1,A] + U[i2,A].
  // The U rows that every row of the tile shares (a row tile of pairs (a<b)
  // mostly shares b, of (i, a<b) shares i and b) are summed once per column
  // into y_A = e_A + U[s1,A] + U[s2,A] - U[i1,A] - U[i2,A] over those slots;
  // each coupling then adds only its row's own rows: D_K = (E0' - chi(e)) - y_A - ...
  const double e0p = *E0p;
  const int64_t mend = adj.T ? adj.m_base + adj.Mc : M;
  __shared__ double sY[GBN];
  int cm = 0;  // bit k: slot k (s1, s2, i1, i2) is the same in every row of the tile
  {
    const RowInfo r0 = rows[m0];
    const int64_t rr = m0 + tid;
    const bool own = tid < GBM && rr < mend;
    const RowInfo ri = own ? rows[rr] : r0;
    cm |= __syncthreads_and(ri.s1 == r0.s1) ? 1 : 0;
    cm |= __syncthreads_and(ri.s2 == r0.s2) ? 2 : 0;
    cm |= __syncthreads_and(ri.i1 == r0.i1) ? 4 : 0;
    cm |= __syncthreads_and(ri.i2 == r0.i2) ? 8 : 0;
    if (tid < GBN) {
      const int64_t col = sCol[tid];
      double y = 0.0;
      if (col >= 0) {
        y = eA[col];
        if (cm & 1) y += U[(int64_t)r0.s1 * N + col];
        if (cm & 2) y += U[(int64_t)r0.s2 * N + col];
        if (cm & 4) y -= U[(int64_t)r0.i1 * N + col];
        if (cm & 8) y -= U[(int64_t)r0.i2 * N + col];
      }
      sY[tid] = y;
    }
    __syncthreads();
  }
  double acc = 0.0, acc2 = 0.0;
  const double inv_n = adj.T ? 1.0 / adj.g1[0].x : 0.0, s2n = 2.0 * adj.s * inv_n;
  unsigned long long dm = ~0ULL;                                // smallest |D| key of the thread
  double rowp[2][2] = {{0.0, 0.0}, {0.0, 0.0}};                 // adjoint: per-row sums of df/dD
  double colp[2][2] = {{0.0, 0.0}, {0.0, 0.0}};                 // adjoint: per-column sums of df/dD
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int64_t row = m0 + wm * 32 + mi * 16 + g + hr * 8;
      if (row >= mend) continue;
      const RowInfo ri = rows[row];
      const double* U1 = U + (int64_t)ri.s1 * N;
      const double* U2 = U + (int64_t)ri.s2 * N;
      const double* U3 = U + (int64_t)ri.i1 * N;
      const double* U4 = U + (int64_t)ri.i2 * N;
      const double base = e0p - ri.chi;
      const bool in_q = ri.chi != kExcludedChi;  // external subspace limits
      // the thread's four denominators of this row, inverted together
      double Dv[4], q[4], rq[4];
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int hc = 0; hc < 2; ++hc) {
          const int lc = wn * 16 + ni * 8 + 2 * tq + hc;
          const int64_t col = sCol[lc];
          const int kk = ni * 2 + hc;
          if (col >= 0) {  // tile-uniform branches
            double d = base - sY[lc];
            if (!(cm & 1)) d -= U1[col];
            if (!(cm & 2)) d -= U2[col];
            if (!(cm & 4)) d += U3[col];
            if (!(cm & 8)) d += U4[col];
            Dv[kk] = d;
          } else {
            Dv[kk] = 1.0;
          }
          q[kk] = col >= 0 ? en_q(Dv[kk], b) : 1.0;
          if (col >= 0 && in_q) dm = min(dm, dkey(Dv[kk]));
        }
      rcp4(q, rq);
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int hc = 0; hc < 2; ++hc) {
          const int64_t col = sCol[wn * 16 + ni * 8 + 2 * tq + hc];
          const int64_t slot = adj.t_tile ? (row - adj.m_base) * adj.t_ld + n0 + wn * 16 + ni * 8 + 2 * tq + hc
                                          : (row - adj.m_base) * N + col;
          if (col < 0) {
            if (adj.T && adj.t_tile) {  // padding column of a tile-ordered amplitude row
              adj.T[slot] = make_double2(0.0, 0.0);
              if (adj.Hm) adj.Hm[slot] = 0.0;
            }
            continue;
          }
          const int e = hr * 2 + hc, kk = ni * 2 + hc;
          const double vr = t1[mi][ni][e] - t2[mi][ni][e];
          const double vi = t3[mi][ni][e] - t1[mi][ni][e] - t2[mi][ni][e];
          const double Dk = Dv[kk];
          const double v2 = fma(vr, vr, vi * vi);
          if (!adj.T) {
            acc = fma(v2, en_g_r(Dk, b, rq[kk]), acc);  // the E2 term, same rounding in both passes
            if (adj.probeV) {
              const int lr = wm * 32 + mi * 16 + g + hr * 8, lc = wn * 16 + ni * 8 + 2 * tq + hc;
              adj.probeV[lr * GBN + lc] = make_double2(vr, vi);
              adj.probeD[lr * GBN + lc] = Dk;
            }
          } else {
            double gk, hk;
            en_derivs_r(v2 * inv_n, Dk, b, rq[kk], gk, hk);
            const double w = s2n * gk;  // t = s (2/n) g V
            adj.T[slot] = make_double2(w * vr, w * vi);
            hk *= adj.s;
            if (adj.Hm) adj.Hm[slot] = hk;
            rowp[mi][hr] += hk;
            colp[ni][hc] += hk;
            acc += hk;
            acc2 = fma(v2, gk, acc2);  // the forward's E2 term (gk = en_g_r(Dk, b, r))
          }
        }
    }
  dmin_flush(dmin, dm);
  if (adj.T) {
    // fixed-order per-row / per-column sums over the tile (16 contributors each)
    __shared__ double sRow[GBM][16], sColP[GBN][16];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int hr = 0; hr < 2; ++hr) sRow[wm * 32 + mi * 16 + g + hr * 8][wn * 4 + tq] = rowp[mi][hr];
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int hc = 0; hc < 2; ++hc) sColP[wn * 16 + ni * 8 + 2 * tq + hc][wm * 8 + g] = colp[ni][hc];
    __syncthreads();
    if (tid < GBM) {
      double s = 0.0;
      for (int k = 0; k < 16; ++k) s += sRow[tid][k];
      const int64_t row = m0 + tid;
      if (row < mend) adj.Hrow[(row - adj.m_base) * n_tile_n + tile_n] = s;  // chunk-local rows
    } else if (tid < GBM + GBN) {
      const int c = tid - GBM;
      double s = 0.0;
      for (int k = 0; k < 16; ++k) s += sColP[c][k];
      const int64_t col = sCol[c];
      if (col >= 0) adj.Hcol[tile_m * N + col] = s;  // chunk-local row tiles
    }
    const double fs = block_sum(acc2, sh);  // sum f over the tile, as the forward sums it
    const double t2s = adj.s * inv_n * fs;  // sum s (df/dv) v
    double ts = block_sum(acc, sh);
    if (tid == 0) {
      const int64_t slot = tile_m * n_tile_n + tile_n;  // chunk-local
      adj.scal[2 * slot] = ts;
      adj.scal[2 * slot + 1] = t2s;
    }
    if (adj.part && tid == 0)  // the forward's partial of this tile, same terms in the same order
      adj.part[tile_n * adj.rt + (adj.m_base / GBM) + tile_m] = fs;
    return;
  }
  double tot = block_sum(acc, sh);
  if (tid == 0) *partial_slot = tot;
}

// Compacted coupling table of a column-tiled class (one block per tile):
//   Dc[(koff + k) * 64 + c] = D[klist[koff + k]][perm[64 j + c]], 0 beyond ktrue or for padding
__global__ void k_dcompact(const double2* __restrict__ D, int64_t N, ColTiles ctl, double2* __restrict__ Dc) {
  const int j = blockIdx.x;
  const int4 td = ctl.tdesc[j];
  for (int i = threadIdx.x; i < td.y * GBN; i += blockDim.x) {
    const int kk = i / GBN, c = i % GBN;
    const int32_t p = ctl.perm[(int64_t)j * GBN + c];
    double2 v = make_double2(0.0, 0.0);
    if (kk < td.z && p >= 0) v = D[(int64_t)ctl.klist[td.x + kk] * N + p];
    Dc[((int64_t)td.x + kk) * GBN + c] = v;
  }
}

// One CTA per 64x64 tile: gridDim.x row tiles (of the chunk from adj.m_base,
// or tm0 .. tm0 + gridDim.x - 1 of the rt the class has: a shard, or all)
// times gridDim.y column tiles.  Forward: one partial per tile, in
// partial[column tile * rt + row tile].
// Rasterisation in bands of row tiles: the CTAs in flight share a band's
// integral rows (W, 64 rows x Kp each), which stay in L2 while the band
// sweeps every column tile, so W is read from DRAM about once instead of
// once per column tile (at the Ar shape 0.36 GB against 686 GB for class
// (0,2)); the coupling-table blocks and the epilogue's U rows are read once
// per band.  A band holds about 24 MiB of W (8 to 512 row tiles).
__device__ __forceinline__ int64_t class_band(int Kp) {
  const int64_t b = ((int64_t)24 << 20) / ((int64_t)GBM * 16 * Kp);
  return b < 8 ? 8 : b > 512 ? 512 : b;
}
__global__ void __launch_bounds__(256, 1)
k_class_gemm(const double2* __restrict__ W, const double2* __restrict__ D, int64_t M, int64_t N, int Kp,
             const RowInfo* __restrict__ rows, const double* __restrict__ U, const double* __restrict__ eA,
             const double* __restrict__ E0p, double b, double* __restrict__ partial, AdjOut adj, ColTiles ctl,
             unsigned long long* dmin, int64_t rt, int64_t tm0) {
  const int64_t gx = gridDim.x, gy = gridDim.y, kB = class_band(Kp);
  const int64_t L = (int64_t)blockIdx.y * gx + blockIdx.x;  // launch order
  const int64_t band = L / (kB * gy), b0 = band * kB;
  const int64_t bsz = gx - b0 < kB ? gx - b0 : kB;          // the last band may be narrower
  const int64_t r = L - b0 * gy;
  const int64_t tm = tm0 + b0 + r % bsz, tn = r / bsz;
  double* slot = partial ? partial + tn * rt + tm : nullptr;
  class_tile(W, D, M, N, Kp, rows, U, eA, E0p, b, slot, adj, tm, tn, gy, ctl, dmin);
}

// One tile (tile_m, tile_n) of the class kernel with its per-coupling probe
// outputs set (adj.probeV / probeD): the same device code as k_class_gemm.
__global__ void __launch_bounds__(256, 1)
k_class_probe(const double2* __restrict__ W, const double2* __restrict__ D, int64_t M, int64_t N, int Kp,
              const RowInfo* __restrict__ rows, const double* __restrict__ U, const double* __restrict__ eA,
              const double* __restrict__ E0p, double b, double* __restrict__ partial, AdjOut adj, ColTiles ctl,
              int64_t tile_m, int64_t tile_n, int64_t n_tile_n) {
  class_tile(W, D, M, N, Kp, rows, U, eA, E0p, b, partial, adj, tile_m, tile_n, n_tile_n, ctl, nullptr);
}

// ------------------------------------------------------------------ class (2,2)

// sum_{i<j, a<b, A} |<ab||ij>|^2 |c_A|^2 / D  with
// D = E0' - e_A + U[i,A] + U[j,A] - chi_ij - (alpha_a + U[a,A]) - (alpha_b + U[b,A]) - G_ab,
// chi_ij = -eps^_i - eps^_j + G_ij, alpha_a = eps^_a - G_ia - G_ja.
// Grid: x = A tiles (one A per thread), y = ordered pairs of 8-wide virtual
// blocks, z = (i<j).  One partial per CTA.
// One block (string tile bx of gx, unit u) of the class; the kernel below and
// the persistent batch kernel run it with the same partial slot.
__device__ __forceinline__ void class22_block(const DevList& Ls, const DevSpace& sp, const double2* __restrict__ c,
                                              const double* __restrict__ g2, const double* __restrict__ epsh,
                                              const double* __restrict__ G, const double* __restrict__ E0p, double b,
                                              int nvb, double* __restrict__ partial, unsigned long long* dmin,
                                              int64_t u, int64_t bx, int64_t gx) {
  __shared__ double sGab[8][8], sG2[8][8], sAl[2][8];
  __shared__ double sh[32];
  // unit u = (core pair z, virtual block pair y), u = z nyb + y
  const int64_t nyb = (int64_t)nvb * (nvb + 1) / 2;
  const int zp = (int)(u / nyb);
  int ba = 0, bb = 0;
  {
    int yb = (int)(u % nyb), k = 0;
    while (yb >= nvb - k) { yb -= nvb - k; ++k; }
    ba = k;
    bb = k + yb;
  }
  int iu, ju;
  pair_decode(zp, iu, ju);
  const int gi = sp.cc[iu], gj = sp.cc[ju];
  const int64_t nvp = pairs(sp.nvc);
  const int tid = threadIdx.x;
  if (tid < 64) {
    int x = tid >> 3, y = tid & 7;
    int a = ba * 8 + x, bq = bb * 8 + y;
    bool ok = a < sp.nvc && bq < sp.nvc && a < bq;
    sGab[x][y] = ok ? G[(int64_t)sp.vc[a] * sp.n + sp.vc[bq]] : 0.0;
    sG2[x][y] = ok ? g2[(int64_t)zp * nvp + pair_index(a, bq)] : 0.0;
  } else if (tid < 80) {
    int k = tid - 64, side = k >> 3, x = k & 7;
    int a = (side ? bb : ba) * 8 + x;
    double al = 0.0;
    if (a < sp.nvc) {
      int ga = sp.vc[a];
      al = epsh[ga] - G[(int64_t)gi * sp.n + ga] - G[(int64_t)gj * sp.n + ga];
    }
    sAl[side][x] = al;
  }
  __syncthreads();
  const int64_t A = bx * (int64_t)blockDim.x + tid;
  double acc = 0.0;
  unsigned long long dm = ~0ULL;
  if (A < Ls.n) {
    const double chi_ij = -epsh[gi] - epsh[gj] + G[(int64_t)gi * sp.n + gj];
    const double ct = *E0p - Ls.eA[A] + Ls.U[(int64_t)iu * Ls.n + A] + Ls.U[(int64_t)ju * Ls.n + A] - chi_ij;
    double pa[8], pb[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      int a = ba * 8 + k, bq = bb * 8 + k;
      pa[k] = (a < sp.nvc) ? sAl[0][k] + Ls.U[(int64_t)(sp.ncc + a) * Ls.n + A] : 0.0;
      pb[k] = (bq < sp.nvc) ? sAl[1][k] + Ls.U[(int64_t)(sp.ncc + bq) * Ls.n + A] : 0.0;
    }
    double inner = 0.0;
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      const double cx = ct - pa[x];
#pragma unroll
      for (int y0 = 0; y0 < 8; y0 += 4) {  // four denominators inverted together
        double Dv[4], q[4], rq[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          Dv[k] = cx - pb[y0 + k] - sGab[x][y0 + k];
          q[k] = sG2[x][y0 + k] != 0.0 ? en_q(Dv[k], b) : 1.0;
          if (sG2[x][y0 + k] != 0.0) dm = min(dm, dkey(Dv[k]));  // the couplings the sum takes
        }
        rcp4(q, rq);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double w = sG2[x][y0 + k];
          if (w != 0.0) inner = fma(w, en_g_r(Dv[k], b, rq[k]), inner);
        }
      }
    }
    double2 cv = c[A];
    acc = fma(cv.x, cv.x, cv.y * cv.y) * inner;
  }
  dmin_flush(dmin, dm);
  double tot = block_sum(acc, sh);
  if (tid == 0) partial[u * gx + bx] = tot;
}

// Grid: x = A tiles (one A per thread), y = units u0 + blockIdx.y.  One partial per CTA.
__global__ void __launch_bounds__(256)
k_class22(DevList Ls, DevSpace sp, const double2* __restrict__ c, const double* __restrict__ g2 /*[ncp][nvp]*/,
          const double* __restrict__ epsh, const double* __restrict__ G, const double* __restrict__ E0p, double b,
          int nvb, double* __restrict__ partial, unsigned long long* dmin, int64_t u0) {
  class22_block(Ls, sp, c, g2, epsh, G, E0p, b, nvb, partial, dmin, u0 + blockIdx.y, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------ gather classes

// (0,1): V[a,A] = sum_t f_at D^t_A + sum_{u in A} (-1)^{#A<u} sum_{v<w} <au||vw> D^{vw}_{A-u}
// One block (string tile bx of gx, virtual a) of the class.
__device__ __forceinline__ void class01_block(const DevList& L01, const DevList& L12, const DevList& L02,
                                              const DevDas& das, const DevSpace& sp, const int64_t* __restrict__ binom,
                                              const double2* __restrict__ DT, const double2* __restrict__ DTU,
                                              const double2* __restrict__ X01, const double2* __restrict__ f,
                                              const double* __restrict__ epsh, const double* __restrict__ E0p,
                                              double b, double* __restrict__ partial, unsigned long long* dmin,
                                              double2* __restrict__ probeV, double* __restrict__ probeD, int a,
                                              int64_t bx, int64_t gx) {
  __shared__ double sh[32];
  const int64_t g = bx * (int64_t)blockDim.x + threadIdx.x;
  const int na = sp.n_act, ntp = (int)pairs(na);
  double acc = 0.0;
  unsigned long long dm = ~0ULL;
  if (g < L01.n) {
    const uint64_t A = L01.str[g];
    const int ga = sp.vc[a];
    double2 V = make_double2(0.0, 0.0);
    int64_t a12 = list_addr(L12, das, binom, A);
    if (a12 >= 0)
      for (int t = 0; t < na; ++t) V = cfma(f[(int64_t)ga * sp.n_occ + sp.a0 + t], DT[(int64_t)t * L12.n + a12], V);
    for (uint64_t x = A; x; x &= x - 1) {
      const int u = __ffsll((long long)x) - 1;
      const uint64_t B = A & ~(1ull << u);
      const int64_t a02 = list_addr(L02, das, binom, B);
      if (a02 < 0) continue;
      double2 s = make_double2(0.0, 0.0);
      const double2* Xr = X01 + ((int64_t)a * na + u) * ntp;
      for (int w = 1; w < na; ++w) {
        if ((B >> w) & 1) continue;
        for (int v = 0; v < w; ++v) {
          if ((B >> v) & 1) continue;
          const int vw = pair_index(v, w);
          s = cfma(Xr[vw], DTU[(int64_t)vw * L02.n + a02], s);
        }
      }
      if (popc_below(A, u) & 1) s = make_double2(-s.x, -s.y);
      V.x += s.x;
      V.y += s.y;
    }
    const double Dk = *E0p - L01.eA[g] - epsh[ga] - L01.U[(int64_t)(sp.ncc + a) * L01.n + g];
    acc = fma(V.x, V.x, V.y * V.y) * en_g(Dk, b);
    dm = dkey(Dk);
    if (probeV) {  // per-coupling check: row (blockIdx.y) x string
      probeV[(int64_t)a * L01.n + g] = V;
      probeD[(int64_t)a * L01.n + g] = Dk;
    }
  }
  dmin_flush(dmin, dm);
  double tot = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[(int64_t)a * gx + bx] = tot;
}

// grid x: string tiles, y: virtuals u0 + blockIdx.y (a shard, or all)
__global__ void k_class01(DevList L01, DevList L12, DevList L02, DevDas das, DevSpace sp, const int64_t* __restrict__ binom,
                          const double2* __restrict__ DT /*[KpT][n12]*/, const double2* __restrict__ DTU /*[KpTU][n02]*/,
                          const double2* __restrict__ X01, const double2* __restrict__ f, const double* __restrict__ epsh,
                          const double* __restrict__ E0p, double b, double* __restrict__ partial, unsigned long long* dmin,
                          double2* __restrict__ probeV, double* __restrict__ probeD, int64_t u0) {
  class01_block(L01, L12, L02, das, sp, binom, DT, DTU, X01, f, epsh, E0p, b, partial, dmin, probeV, probeD,
                (int)(u0 + blockIdx.y), blockIdx.x, gridDim.x);
}

// (1,0): V[i,A] = sum_t f_ti D^{t+}_A + sum_{t<u in A} s(A;t,u) sum_v <tu||iv> D^v_{A-t-u}
// One block (string tile bx of gx, core spinor i) of the class.
__device__ __forceinline__ void class10_block(const DevList& L10, const DevList& L21, const DevList& L12,
                                              const DevDas& das, const DevSpace& sp, const int64_t* __restrict__ binom,
                                              const double2* __restrict__ DTD, const double2* __restrict__ DT,
                                              const double2* __restrict__ X10, const double2* __restrict__ f,
                                              const double* __restrict__ epsh, const double* __restrict__ E0p,
                                              double b, double* __restrict__ partial, unsigned long long* dmin,
                                              double2* __restrict__ probeV, double* __restrict__ probeD, int i,
                                              int64_t bx, int64_t gx) {
  __shared__ double sh[32];
  const int64_t g = bx * (int64_t)blockDim.x + threadIdx.x;
  const int na = sp.n_act;
  double acc = 0.0;
  unsigned long long dm = ~0ULL;
  if (g < L10.n) {
    const uint64_t A = L10.str[g];
    const int gi = sp.cc[i];
    double2 V = make_double2(0.0, 0.0);
    int64_t a21 = list_addr(L21, das, binom, A);
    if (a21 >= 0)
      for (int t = 0; t < na; ++t) V = cfma(f[(int64_t)(sp.a0 + t) * sp.n_occ + gi], DTD[(int64_t)t * L21.n + a21], V);
    for (uint64_t xu = A; xu; xu &= xu - 1) {
      const int u = __ffsll((long long)xu) - 1;
      for (uint64_t xt = A & ((1ull << u) - 1); xt; xt &= xt - 1) {
        const int t = __ffsll((long long)xt) - 1;
        const uint64_t B = A & ~(1ull << t) & ~(1ull << u);
        const int64_t a12 = list_addr(L12, das, binom, B);
        if (a12 < 0) continue;
        const double2* Xr = X10 + ((int64_t)i * pairs(na) + pair_index(t, u)) * na;
        double2 s = make_double2(0.0, 0.0);
        for (int v = 0; v < na; ++v) {
          if ((B >> v) & 1) continue;
          s = cfma(Xr[v], DT[(int64_t)v * L12.n + a12], s);
        }
        if ((popc_below(B, u) + popc_below(B, t)) & 1) s = make_double2(-s.x, -s.y);
        V.x += s.x;
        V.y += s.y;
      }
    }
    const double Dk = *E0p - L10.eA[g] + epsh[gi] + L10.U[(int64_t)i * L10.n + g];
    acc = fma(V.x, V.x, V.y * V.y) * en_g(Dk, b);
    dm = dkey(Dk);
    if (probeV) {  // per-coupling check: row (blockIdx.y) x string
      probeV[(int64_t)i * L10.n + g] = V;
      probeD[(int64_t)i * L10.n + g] = Dk;
    }
  }
  dmin_flush(dmin, dm);
  double tot = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[(int64_t)i * gx + bx] = tot;
}

// grid x: string tiles, y: core spinors u0 + blockIdx.y (a shard, or all)
__global__ void k_class10(DevList L10, DevList L21, DevList L12, DevDas das, DevSpace sp, const int64_t* __restrict__ binom,
                          const double2* __restrict__ DTD /*[Kp][n21]*/, const double2* __restrict__ DT /*[Kp][n12]*/,
                          const double2* __restrict__ X10, const double2* __restrict__ f, const double* __restrict__ epsh,
                          const double* __restrict__ E0p, double b, double* __restrict__ partial, unsigned long long* dmin,
                          double2* __restrict__ probeV, double* __restrict__ probeD, int64_t u0) {
  class10_block(L10, L21, L12, das, sp, binom, DTD, DT, X10, f, epsh, E0p, b, partial, dmin, probeV, probeD,
                (int)(u0 + blockIdx.y), blockIdx.x, gridDim.x);
}

// (0,0), DAS only: V[A] = <A|H - E_O|Psi> for A of a non-reference pattern
// One block (string block blk) of the class.
__device__ __forceinline__ void class00_block(const DevList& L00, const DevList& L11, const DevList& L02,
                                              const DevDas& das, const DevSpace& sp, const int64_t* __restrict__ binom,
                                              const double2* __restrict__ DTDU, const double2* __restrict__ DTU,
                                              const double2* __restrict__ X00, const double2* __restrict__ f,
                                              const double* __restrict__ E0p, double b, double* __restrict__ partial,
                                              unsigned long long* dmin, double2* __restrict__ probeV,
                                              double* __restrict__ probeD, int64_t blk) {
  __shared__ double sh[32];
  const int64_t g = blk * (int64_t)blockDim.x + threadIdx.x;
  double acc = 0.0;
  unsigned long long dm = ~0ULL;
  if (g < L00.n) {
    const double2 V = active_sigma(L00.str[g], L11, L02, das, sp, binom, DTDU, DTU, X00, f);
    const double Dk = *E0p - L00.eA[g];
    acc = fma(V.x, V.x, V.y * V.y) * en_g(Dk, b);
    dm = dkey(Dk);
    if (probeV) {  // per-coupling check: row (blockIdx.y) x string
      probeV[g] = V;
      probeD[g] = Dk;
    }
  }
  dmin_flush(dmin, dm);
  double tot = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blk] = tot;
}

// grid x: string blocks u0 + blockIdx.x (a shard, or all)
__global__ void k_class00(DevList L00, DevList L11, DevList L02, DevDas das, DevSpace sp, const int64_t* __restrict__ binom,
                          const double2* __restrict__ DTDU /*[Kp][n11]*/, const double2* __restrict__ DTU /*[Kp][n02]*/,
                          const double2* __restrict__ X00, const double2* __restrict__ f, const double* __restrict__ E0p,
                          double b, double* __restrict__ partial, unsigned long long* dmin,
                          double2* __restrict__ probeV, double* __restrict__ probeD, int64_t u0) {
  class00_block(L00, L11, L02, das, sp, binom, DTDU, DTU, X00, f, E0p, b, partial, dmin, probeV, probeD,
                u0 + blockIdx.x);
}

// ------------------------------------------------------------------ persistent batch launch

// One launch for every class of every (job, root) of a batch: one CTA per SM
// takes work items from an integer counter.  The items form runs (WorkSeg) of
// one kind each: the 64 x 64 tiles of a dense class, or the blocks of class
// (2,2) or of a gather class; runs are ordered longest item first, so that
// the short (2,2) blocks fill the tail.  Every item writes the same partial
// slot as the one-launch-per-class form, so the reduction order is unchanged
// and the energies are bitwise those of e2_forward.
__global__ void __launch_bounds__(256, 1)
k_batch(const WorkSeg* __restrict__ segs, int nseg, const GemmJob* __restrict__ gjobs,
        const SparseJob* __restrict__ sjobs, int64_t total, unsigned long long* __restrict__ counter) {
  __shared__ long long s_item;
  const AdjOut none{};
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t it = s_item;
    if (it >= total) break;
    int lo = 0, hi = nseg - 1;  // the run holding item it
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (segs[mid].first <= it) lo = mid;
      else hi = mid - 1;
    }
    const WorkSeg w = segs[lo];
    const int64_t k = it - w.first;
    if (w.kind == WORK_TILE) {
      const GemmJob& j = gjobs[w.job];
      const int64_t ntm = (j.M + GBM - 1) / GBM, tm = k / w.gx, tn = k % w.gx;
      class_tile(j.W, j.D, j.M, j.N, j.Kp, j.rows, j.U, j.eA, j.E0p, j.b, j.partial + tn * ntm + tm, none, tm, tn,
                 w.gx, j.ct, j.dmin);
      continue;
    }
    const SparseJob& j = sjobs[w.job];
    if (w.kind == WORK_C22)
      class22_block(j.L8, j.sp, j.c, j.g2, j.epsh, j.G, j.E0p, j.b, j.nvb, j.part[0], j.dmin[0], k / w.gx, k % w.gx,
                    w.gx);
    else if (w.kind == WORK_C01)
      class01_block(j.L1, j.L5, j.L2, j.das, j.sp, j.binom, j.DT, j.DTU, j.X01, j.f, j.epsh, j.E0p, j.b, j.part[1],
                    j.dmin[1], nullptr, nullptr, (int)(k / w.gx), k % w.gx, w.gx);
    else if (w.kind == WORK_C10)
      class10_block(j.L3, j.L7, j.L5, j.das, j.sp, j.binom, j.DTD, j.DT, j.X10, j.f, j.epsh, j.E0p, j.b, j.part[2],
                    j.dmin[2], nullptr, nullptr, (int)(k / w.gx), k % w.gx, w.gx);
    else
      class00_block(j.L0, j.L4, j.L2, j.das, j.sp, j.binom, j.DTDU, j.DTU, j.X00, j.f, j.E0p, j.b, j.part[3],
                    j.dmin[3], nullptr, nullptr, k);
  }
}

// ------------------------------------------------------------------ reference solver

// sigma[g] = <A_g| H - E_O |c> for every reference string (P address order)
__global__ void k_sigma(DevList LP, DevList L11, DevList L02, DevDas das, DevSpace sp, const int64_t* __restrict__ binom,
                        const double2* __restrict__ DTDU, const double2* __restrict__ DTU, const double2* __restrict__ X00,
                        const double2* __restrict__ f, double2* __restrict__ sigma) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= LP.n) return;
  sigma[g] = active_sigma(LP.str[g], L11, L02, das, sp, binom, DTDU, DTU, X00, f);
}

// out[j][A] = (acc ? out[j][A] : 0) + sum_i Y[i*k + j] V[i][A]
__global__ void k_lincomb(const double2* __restrict__ V, int m, int64_t n, const double2* __restrict__ Y, int k, int acc,
                          double2* __restrict__ out) {
  const int64_t A = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (A >= n) return;
  double2 s = acc ? out[(int64_t)j * n + A] : make_double2(0.0, 0.0);
  for (int i = 0; i < m; ++i) s = cfma(Y[i * k + j], V[(int64_t)i * n + A], s);
  out[(int64_t)j * n + A] = s;
}

// r <- r - theta x ; then d = r / (theta - diag), |theta - diag| floored at 1e-4
__global__ void k_residual(double2* __restrict__ r, const double2* __restrict__ x, const double* __restrict__ diag,
                           int64_t n, double theta, double2* __restrict__ d) {
  const int64_t A = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (A >= n) return;
  double2 v = r[A], xv = x[A];
  v.x -= theta * xv.x;
  v.y -= theta * xv.y;
  r[A] = v;
  double den = theta - diag[A];
  if (fabs(den) < 1e-4) den = den < 0 ? -1e-4 : 1e-4;
  d[A] = make_double2(v.x / den, v.y / den);
}

__global__ void k_scale(double2* __restrict__ x, int64_t n, double s) {
  const int64_t A = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (A < n) x[A] = make_double2(x[A].x * s, x[A].y * s);
}

// ------------------------------------------------------------------ FP64 peaks

// Independent mma.sync m16n8k8 f64 chains (4 per warp), iters steps each.
__global__ void k_peak_dmma(double* out, int iters) {
  double a[4], bb[2], c[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) a[j] = 1e-3 * (threadIdx.x + j);
  bb[0] = 0.5;
  bb[1] = 0.25;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) c[j][e] = 0.0;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) mma_f64(c[j], a, bb);
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) s += c[j][0] + c[j][1] + c[j][2] + c[j][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Eight independent FP64 FMA chains per thread, iters steps each.
__global__ void k_peak_dfma(double* out, int iters) {
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 1e-3 * (threadIdx.x + j);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], 0.999, 1e-3);
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ------------------------------------------------------------------ reductions

// E2_class[root][cls] = sum of the class partials in index order (one block each);
// norm = <c|c> divides every term (Sec. 2.3 takes Psi normalised).
__global__ void k_reduce(const double* __restrict__ partial, const int64_t* __restrict__ off, const int64_t* __restrict__ cnt,
                         const double2* __restrict__ g1_all, int g1_stride, int n_roots, double* __restrict__ e2c) {
  __shared__ double sh[32];
  const int root = blockIdx.x / E2_NCLASS, cls = blockIdx.x % E2_NCLASS;
  const int64_t o = off[root * E2_NCLASS + cls], n = cnt[cls];
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) acc += partial[o + k];
  double tot = block_sum(acc, sh);
  if (threadIdx.x == 0) e2c[root * E2_NCLASS + cls] = tot / g1_all[(int64_t)root * g1_stride].x;
}

// Status word before a pass: no flags; every smallest-|D| key at the largest
// non-negative int64 (keys stay ordered as signed integers, so ranks can take
// their minimum with a signed reduction).
__global__ void k_status_init(unsigned long long* status, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) status[k] = k ? 0x7FFFFFFFFFFFFFFFULL : 0ULL;
}

// E2 of each root from its class sums, and the device-detected conditions
// into the status word (status[0] flags, status[1 + 9 r + cls] the smallest
// |D| key of the class): a non-finite energy sets ST_NONFINITE; with b = 0 a
// denominator below kIntruderD sets ST_INTRUDER (an intruder state, Sec. 2.6).
__global__ void k_finalize(const double* __restrict__ e2c, int n_roots, double* __restrict__ E2,
                           const double* __restrict__ E0in, double* __restrict__ E0out,
                           unsigned long long* __restrict__ status, double b) {
  int r = threadIdx.x;
  if (r >= n_roots) return;
  double s = 0.0;
  bool bad = false;
  for (int k = 0; k < E2_NCLASS; ++k) {
    const double v = e2c[r * E2_NCLASS + k];
    bad = bad || !isfinite(v);
    s += v;
  }
  E2[r] = s;
  if (E0out) E0out[r] = E0in[r];
  if (!status) return;
  unsigned long long f = (bad || !isfinite(s)) ? ST_NONFINITE : 0ULL;
  if (b == 0.0)
    for (int k = 0; k < E2_NCLASS; ++k)
      if (status[1 + r * E2_NCLASS + k] < dkey(kIntruderD)) f |= ST_INTRUDER;
  if (f) atomicOr(status, f);
}

}  // namespace e2
