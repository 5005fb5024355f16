// sm_103a adjoint kernels of the Epstein-Nesbet second-order energy.
//
// With v_K = |V_K|^2/n (n = <c|c>), D_K = E0 - H_KK, E2 = sum_K f(v_K, D_K),
// f = v/D or, with the level shift of Sec. 2.6, v D^3/(D^4 + b^2), and the
// seed s of the root:
//   t_K = s (2/n) (df/dv) V_K            weighted first-order amplitude
//   eta_K = s df/dD                      denominator weight
//   dE2 = Re sum_K conj(t_K) <K|dH|c> + (sum eta / n) <c|dH|c> - sum_K eta_K <K|dH|K>
//   cbar = H_PQ t - (2/n) s (sum (df/dv) v) c + (2/n) (sum eta) (H_PP - E0) c
// Coefficients Gamma_X below are "dE2 = Re sum Gamma_X dX"; a gradient with
// respect to a complex input z is conj(Gamma_z) (dE2/dRe z + i dE2/dIm z).
#include <cuda_runtime.h>

#include "e2_common.cuh"
#include "e2_device.cuh"
#include "e2_kernels.cuh"
#include "e2_host.h"

namespace e2 {

// ------------------------------------------------------------------ generic complex GEMM

// C(m,n) = beta * C(m,n) + sum_k opA(m,k) opB(k,n) on the FP64 tensor pipe
// (three real products per complex product), opA(m,k) = A[m*sam + k*sak]
// (conjugated when conjA), opB(k,n) = B[k*sbk + n*sbn] (conjugated when
// conjB), C(m,n) = C[m*csm + n*csn].  Tile BM x BN with WM x (8 / WM) warps:
// 64 x 64 (warp tiles 32 x 16), 128 x 16 (warp tiles 16 x 16, for the
// 16-wide outputs of the classes whose contraction is one active index) or
// 64 x 80 (warp tiles 16 x 40, for the compacted rows of a column tile,
// mostly 78 of them for D^{tu} at 16 active spinors).  Split K:
// grid.z segments of kseg, segment z writing C + z*czs (beta applies to each
// segment's own output); a fixed-order sum of the segments (k_zacc) keeps the
// result deterministic.  Each output element is owned by one CTA per segment.
// With lower >= 0 only tiles holding some n <= lower + m are computed.
// Optional index maps gather operand rows / columns: A(m,k) reads row
// amap[m] and column akmap[k] of A, B(k,n) reads column bmap[n] of B; a
// negative map entry reads zero.  (bx, by, bz) = (M tile, N tile, K segment).
template <int BM, int BN, int WM>
__device__ __forceinline__ void zgemm_body(int64_t M, int64_t N, int64_t K, const double2* __restrict__ A, int64_t sam,
                                           int64_t sak, int conjA, const double2* __restrict__ B, int64_t sbk,
                                           int64_t sbn, int conjB, double2* __restrict__ C, int64_t csm, int64_t csn,
                                           int beta, int64_t kseg, int64_t czs, int64_t lower, int64_t bx, int64_t by,
                                           int64_t bz, const int32_t* __restrict__ amap = nullptr,
                                           const int32_t* __restrict__ akmap = nullptr,
                                           const int32_t* __restrict__ bmap = nullptr) {
  constexpr int BK = 8;
  constexpr int WN = 8 / WM;                            // warps across N (WM across M)
  constexpr int MI = BM / (WM * 16);                    // m16 tiles per warp
  constexpr int NI = BN / (WN * 8);                     // n8 tiles per warp
  static_assert(MI >= 1 && NI >= 1 && WM * 16 * MI == BM && WN * 8 * NI == BN, "tile shape");
  __shared__ double sAr[BM][BK + 1], sAi[BM][BK + 1], sAs[BM][BK + 1];
  __shared__ double sBr[BK][BN + 1], sBi[BK][BN + 1], sBs[BK][BN + 1];
  const int64_t m0 = bx * BM, n0 = by * BN;
  if (lower >= 0 && n0 > lower + m0 + BM - 1) return;  // tile above the diagonal n = lower + m
  const int64_t kb0 = bz * kseg, kb1 = kb0 + kseg < K ? kb0 + kseg : K;
  C += bz * czs;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int wm = warp / WN, wn = warp % WN;
  double t1[MI][NI][4], t2[MI][NI][4], t3[MI][NI][4];
#pragma unroll
  for (int a = 0; a < MI; ++a)
#pragma unroll
    for (int c = 0; c < NI; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e) t1[a][c][e] = t2[a][c][e] = t3[a][c][e] = 0.0;
  // load maps follow the contiguous operand dimension: A rows fastest when
  // sam == 1 (else k fastest), B columns fastest unless sbk == 1
  constexpr int NA = BM * BK / 256;          // A elements per thread
  constexpr int NB = (BK * BN + 255) / 256;  // B elements per thread (16 wide: on half the threads)
  const bool a_mfast = (sam == 1 && sak != 1), b_kfast = (sbk == 1 && sbn != 1);
  int ra[NA], ka[NA], rb[NB], kb_[NB];
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    const int e = tid + 256 * q;
    ra[q] = a_mfast ? e % BM : e / BK;
    ka[q] = a_mfast ? e / BM : e % BK;
  }
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int e = tid + 256 * q;
    rb[q] = b_kfast ? e / BK : e % BN;
    kb_[q] = b_kfast ? e % BK : e / BN;
  }
  const double2 zero = make_double2(0.0, 0.0);
  auto ldA = [&](int64_t k0, int q) {
    const int64_t m = m0 + ra[q], k = k0 + ka[q];
    double2 v = zero;
    if (m < M && k < kb1) {
      const int64_t mi = amap ? (int64_t)amap[m] : m, ki = akmap ? (int64_t)akmap[k] : k;
      if (mi >= 0 && ki >= 0) v = A[mi * sam + ki * sak];
    }
    if (conjA) v.y = -v.y;
    return v;
  };
  auto ldB = [&](int64_t k0, int q) {
    const int64_t kb = k0 + kb_[q], nn = n0 + rb[q];
    double2 u = zero;
    if (tid + 256 * q < BK * BN && kb < kb1 && nn < N) {
      const int64_t ni = bmap ? (int64_t)bmap[nn] : nn;
      if (ni >= 0) u = B[kb * sbk + ni * sbn];
    }
    if (conjB) u.y = -u.y;
    return u;
  };
  // register prefetch of the next K step while the tensor pipe works on this one
  double2 pa[NA], pb[NB];
#pragma unroll
  for (int q = 0; q < NA; ++q) pa[q] = ldA(kb0, q);
#pragma unroll
  for (int q = 0; q < NB; ++q) pb[q] = ldB(kb0, q);
  for (int64_t k0 = kb0; k0 < kb1; k0 += BK) {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      sAr[ra[q]][ka[q]] = pa[q].x;
      sAi[ra[q]][ka[q]] = pa[q].y;
      sAs[ra[q]][ka[q]] = pa[q].x + pa[q].y;
    }
#pragma unroll
    for (int q = 0; q < NB; ++q)
      if (tid + 256 * q < BK * BN) {
        sBr[kb_[q]][rb[q]] = pb[q].x;
        sBi[kb_[q]][rb[q]] = pb[q].y;
        sBs[kb_[q]][rb[q]] = pb[q].x + pb[q].y;
      }
    __syncthreads();
    if (k0 + BK < kb1) {
#pragma unroll
      for (int q = 0; q < NA; ++q) pa[q] = ldA(k0 + BK, q);
#pragma unroll
      for (int q = 0; q < NB; ++q) pb[q] = ldB(k0 + BK, q);
    }
    double br[NI][2], bi[NI][2], bs[NI][2];
#pragma unroll
    for (int ni = 0; ni < NI; ++ni) {
      const int cb = wn * (8 * NI) + ni * 8 + g;
      br[ni][0] = sBr[tq][cb]; br[ni][1] = sBr[tq + 4][cb];
      bi[ni][0] = sBi[tq][cb]; bi[ni][1] = sBi[tq + 4][cb];
      bs[ni][0] = sBs[tq][cb]; bs[ni][1] = sBs[tq + 4][cb];
    }
#pragma unroll
    for (int mi = 0; mi < MI; ++mi) {
      const int r0 = wm * (16 * MI) + mi * 16 + g;
      double a[4];
      a[0] = sAr[r0][tq]; a[1] = sAr[r0 + 8][tq]; a[2] = sAr[r0][tq + 4]; a[3] = sAr[r0 + 8][tq + 4];
#pragma unroll
      for (int ni = 0; ni < NI; ++ni) mma_f64(t1[mi][ni], a, br[ni]);
      a[0] = sAi[r0][tq]; a[1] = sAi[r0 + 8][tq]; a[2] = sAi[r0][tq + 4]; a[3] = sAi[r0 + 8][tq + 4];
#pragma unroll
      for (int ni = 0; ni < NI; ++ni) mma_f64(t2[mi][ni], a, bi[ni]);
      a[0] = sAs[r0][tq]; a[1] = sAs[r0 + 8][tq]; a[2] = sAs[r0][tq + 4]; a[3] = sAs[r0 + 8][tq + 4];
#pragma unroll
      for (int ni = 0; ni < NI; ++ni) mma_f64(t3[mi][ni], a, bs[ni]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < MI; ++mi)
#pragma unroll
    for (int ni = 0; ni < NI; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t row = m0 + wm * (16 * MI) + mi * 16 + g + (e >> 1) * 8;
        const int64_t col = n0 + wn * (8 * NI) + ni * 8 + 2 * tq + (e & 1);
        if (row >= M || col >= N) continue;
        double2 v = make_double2(t1[mi][ni][e] - t2[mi][ni][e], t3[mi][ni][e] - t1[mi][ni][e] - t2[mi][ni][e]);
        double2* out = C + row * csm + col * csn;
        if (beta) {
          v.x += out->x;
          v.y += out->y;
        }
        *out = v;
      }
}

__global__ void __launch_bounds__(256, 1)
k_zgemm64(int64_t M, int64_t N, int64_t K, const double2* __restrict__ A, int64_t sam, int64_t sak, int conjA,
          const double2* __restrict__ B, int64_t sbk, int64_t sbn, int conjB, double2* __restrict__ C, int64_t csm,
          int64_t csn, int beta, int64_t kseg, int64_t czs, int64_t lower) {
  zgemm_body<64, 64, 2>(M, N, K, A, sam, sak, conjA, B, sbk, sbn, conjB, C, csm, csn, beta, kseg, czs, lower,
                        blockIdx.x, blockIdx.y, blockIdx.z);
}

__global__ void __launch_bounds__(256, 1)
k_zgemm16(int64_t M, int64_t N, int64_t K, const double2* __restrict__ A, int64_t sam, int64_t sak, int conjA,
          const double2* __restrict__ B, int64_t sbk, int64_t sbn, int conjB, double2* __restrict__ C, int64_t csm,
          int64_t csn, int beta, int64_t kseg, int64_t czs, int64_t lower) {
  zgemm_body<128, 16, 8>(M, N, K, A, sam, sak, conjA, B, sbk, sbn, conjB, C, csm, csn, beta, kseg, czs, lower,
                         blockIdx.x, blockIdx.y, blockIdx.z);
}

// 24-wide outputs: the classes whose contraction is one active index at 24
// active spinors (a 16-wide tiling computes 32 columns for 24)
__global__ void __launch_bounds__(256, 1)
k_zgemm24(int64_t M, int64_t N, int64_t K, const double2* __restrict__ A, int64_t sam, int64_t sak, int conjA,
          const double2* __restrict__ B, int64_t sbk, int64_t sbn, int conjB, double2* __restrict__ C, int64_t csm,
          int64_t csn, int beta, int64_t kseg, int64_t czs, int64_t lower) {
  zgemm_body<128, 24, 8>(M, N, K, A, sam, sak, conjA, B, sbk, sbn, conjB, C, csm, csn, beta, kseg, czs, lower,
                         blockIdx.x, blockIdx.y, blockIdx.z);
}

// Gamma_D of a column-tiled class in compacted form (tile j = blockIdx.y,
// BN compacted rows per blockIdx.x, K segment blockIdx.z):
//   GDc[(koff + k) * 64 + c] (+)= sum_e conj(T[e][perm[64 j + c]]) W[e][klist[koff + k]]
// (T itself instead of conj(T) when conjT == 0: shifted amplitudes arrive conjugated)
// over the chunk's rows e, as the 64 x klen product of the tile's strings
// with its compacted rows; same split-K segments as the plain product.  The
// product width BN (32, 48, 64 or 80) is the plan's: the one that pads the
// class's compacted lengths least, since every padded row is a full row of
// FP64 tensor work.
template <int BN>
__global__ void __launch_bounds__(256, 1)
k_zgemm_gd_tiles(ColTiles ctl, const double2* __restrict__ W, int Kp, const double2* __restrict__ T, int64_t N,
                 int64_t Mc, double2* __restrict__ GDc, int beta, int64_t kseg, int64_t czs, int conjT,
                 int64_t t_ld) {
  const int j = blockIdx.y;
  const int4 td = ctl.tdesc[j];
  if ((int64_t)blockIdx.x * BN >= td.y) return;
  // T in tile order (t_ld > 0): the tile's 64 columns are contiguous in each row
  const double2* A = t_ld ? T + (int64_t)j * 64 : T;
  zgemm_body<64, BN, 4>(64, td.y, Mc, A, 1, t_ld ? t_ld : N, conjT, W, Kp, 1, 0, GDc + (int64_t)td.x * 64, 1, 64,
                        beta, kseg, czs, -1, 0, blockIdx.x, blockIdx.z,
                        t_ld ? nullptr : ctl.perm + (int64_t)j * 64, nullptr, ctl.klist + td.x);
}

// Gamma_W of a column-tiled class in compacted form (tile j = blockIdx.z):
//   GWc[e * krows + koff + k] = sum_c conj(T[e][perm[64 j + c]]) Dc[(koff + k) * 64 + c]
// (T itself when conjT == 0); product width BN as above.
template <int BN>
__global__ void __launch_bounds__(256, 1)
k_zgemm_gw_tiles(ColTiles ctl, const double2* __restrict__ T, int64_t N, int64_t Mc, int64_t krows,
                 double2* __restrict__ GWc, int conjT, int64_t t_ld) {
  const int j = blockIdx.z;
  const int4 td = ctl.tdesc[j];
  if ((int64_t)blockIdx.y * BN >= td.y) return;
  const double2* A = t_ld ? T + (int64_t)j * 64 : T;  // tile order: contiguous row segments
  zgemm_body<64, BN, 4>(Mc, td.y, 64, A, t_ld ? t_ld : N, 1, conjT, ctl.Dc + (int64_t)td.x * 64, 1, 64, 0,
                        GWc + td.x, krows, 1, 0, 64, 0, -1, blockIdx.x, blockIdx.y, 0, nullptr,
                        t_ld ? nullptr : ctl.perm + (int64_t)j * 64, nullptr);
}

void launch_gd_tiles(int bn, dim3 grid, cudaStream_t st, const ColTiles& ctl, const double2* W, int Kp,
                     const double2* T, int64_t N, int64_t Mc, double2* GDc, int beta, int64_t kseg, int64_t czs,
                     int conjT, int64_t t_ld) {
  switch (bn) {
    case 32: k_zgemm_gd_tiles<32><<<grid, 256, 0, st>>>(ctl, W, Kp, T, N, Mc, GDc, beta, kseg, czs, conjT, t_ld); break;
    case 48: k_zgemm_gd_tiles<48><<<grid, 256, 0, st>>>(ctl, W, Kp, T, N, Mc, GDc, beta, kseg, czs, conjT, t_ld); break;
    case 64: k_zgemm_gd_tiles<64><<<grid, 256, 0, st>>>(ctl, W, Kp, T, N, Mc, GDc, beta, kseg, czs, conjT, t_ld); break;
    default: k_zgemm_gd_tiles<80><<<grid, 256, 0, st>>>(ctl, W, Kp, T, N, Mc, GDc, beta, kseg, czs, conjT, t_ld); break;
  }
  ++g_launches;
}

void launch_gw_tiles(int bn, int64_t Mc, int maxklen, int64_t tiles, cudaStream_t st, const ColTiles& ctl,
                     const double2* T, int64_t N, int64_t krows, double2* GWc, int conjT, int64_t t_ld) {
  const dim3 g((unsigned)((Mc + 63) / 64), (unsigned)((maxklen + bn - 1) / bn), (unsigned)tiles);
  switch (bn) {
    case 32: k_zgemm_gw_tiles<32><<<g, 256, 0, st>>>(ctl, T, N, Mc, krows, GWc, conjT, t_ld); break;
    case 48: k_zgemm_gw_tiles<48><<<g, 256, 0, st>>>(ctl, T, N, Mc, krows, GWc, conjT, t_ld); break;
    case 64: k_zgemm_gw_tiles<64><<<g, 256, 0, st>>>(ctl, T, N, Mc, krows, GWc, conjT, t_ld); break;
    default: k_zgemm_gw_tiles<80><<<g, 256, 0, st>>>(ctl, T, N, Mc, krows, GWc, conjT, t_ld); break;
  }
  ++g_launches;
}

// GD[klist[koff + k]][perm[64 j + c]] += GDc[(koff + k) * 64 + c], k < ktrue (one block per tile)
__global__ void k_gd_scatter(ColTiles ctl, const double2* __restrict__ GDc, int64_t N, double2* __restrict__ GD) {
  const int j = blockIdx.x;
  const int4 td = ctl.tdesc[j];
  for (int i = threadIdx.x; i < td.z * 64; i += blockDim.x) {
    const int k = i / 64, c = i % 64;
    const int32_t p = ctl.perm[(int64_t)j * 64 + c];
    if (p < 0) continue;
    double2* o = GD + (int64_t)ctl.klist[td.x + k] * N + p;
    const double2 v = GDc[((int64_t)td.x + k) * 64 + c];
    o->x += v.x;
    o->y += v.y;
  }
}

// GW[e * ldo + x] = sum_j GWc[e * krows + koff_j + pos[j][x]], x < nxo, over
// the tiles j whose compacted rows include x (pos[j][x] >= 0, pos rows Kp
// wide), in tile order
__global__ void k_gw_reduce(const int4* __restrict__ tdesc, const int32_t* __restrict__ pos, int64_t tiles, int Kp,
                            const double2* __restrict__ GWc, int64_t krows, int64_t Mc, double2* __restrict__ GW,
                            int nxo, int64_t ldo) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= Mc * nxo) return;
  const int64_t e = idx / nxo;
  const int x = (int)(idx % nxo);
  double2 s = make_double2(0.0, 0.0);
  const double2* row = GWc + e * krows;
  for (int64_t j = 0; j < tiles; ++j) {
    const int32_t p = pos[j * Kp + x];
    if (p < 0) continue;
    const double2 v = row[tdesc[j].x + p];
    s.x += v.x;
    s.y += v.y;
  }
  GW[e * ldo + x] = s;
}

// C(m,n) = beta C(m,n) + sum_z part[z*ps + m*N + n] in z order (segments of a
// split-K product, each dense row-major), C(m,n) at C[m*csm + n*csn]
__global__ void k_zacc(const double2* __restrict__ part, int nseg, int64_t ps, int64_t M, int64_t N,
                       double2* __restrict__ C, int64_t csm, int64_t csn, int beta) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M * N) return;
  double2* out = C + (i / N) * csm + (i % N) * csn;
  double2 v = beta ? *out : make_double2(0.0, 0.0);
  for (int z = 0; z < nseg; ++z) {
    const double2 p = part[z * ps + i];
    v.x += p.x;
    v.y += p.y;
  }
  *out = v;
}

// out[i] += sum_z part[z*ps + i] in z order (real split-K segments)
__global__ void k_dacc(const double* __restrict__ part, int nseg, int64_t ps, int64_t count, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  double v = out[i];
  for (int z = 0; z < nseg; ++z) v += part[z * ps + i];
  out[i] = v;
}

// C[m][n] = beta * C[m][n] + sum_k A[m*sam + k*sak] B[k*sbk + n*sbn], real,
// on the FP64 tensor pipe; one CTA per 64x64 tile of C and K segment
// (grid.z segments of kseg, segment z writing C + z*czs).
__global__ void __launch_bounds__(256, 2)
k_dgemm(int64_t M, int64_t N, int64_t K, const double* __restrict__ A, int64_t sam, int64_t sak,
        const double* __restrict__ B, int64_t sbk, int64_t sbn, double* __restrict__ C, int64_t ldc, int beta,
        int64_t kseg, int64_t czs) {
  constexpr int BM = 64, BN = 64, BK = 8;
  __shared__ double sA[BM][BK + 1], sB[BK][BN + 1];
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int64_t kb0 = (int64_t)blockIdx.z * kseg, K1 = kb0 + kseg < K ? kb0 + kseg : K;
  C += (int64_t)blockIdx.z * czs;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int wm = warp >> 2, wn = warp & 3;
  double acc[2][2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[a][c][e] = 0.0;
  const int ar = tid >> 3, ak = tid & 7, bk = tid >> 6, bc = tid & 63;
  for (int64_t k0 = kb0; k0 < K1; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int64_t m = m0 + ar + 32 * q, k = k0 + ak;
      sA[ar + 32 * q][ak] = (m < M && k < K1) ? A[m * sam + k * sak] : 0.0;
      const int64_t kb = k0 + bk + 4 * q, nn = n0 + bc;
      sB[bk + 4 * q][bc] = (kb < K1 && nn < N) ? B[kb * sbk + nn * sbn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
      const int r0 = wm * 32 + mi * 16 + g;
      double a[4] = {sA[r0][tq], sA[r0 + 8][tq], sA[r0][tq + 4], sA[r0 + 8][tq + 4]};
#pragma unroll
      for (int ni = 0; ni < 2; ++ni) {
        const int cb = wn * 16 + ni * 8 + g;
        double b2[2] = {sB[tq][cb], sB[tq + 4][cb]};
        mma_f64(acc[mi][ni], a, b2);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t row = m0 + wm * 32 + mi * 16 + g + (e >> 1) * 8;
        const int64_t col = n0 + wn * 16 + ni * 8 + 2 * tq + (e & 1);
        if (row >= M || col >= N) continue;
        double* out = C + row * ldc + col;
        *out = beta ? *out + acc[mi][ni][e] : acc[mi][ni][e];
      }
}

// Hocc[r][t] = sum_A H[r][A] [t in A]  (one block per row of the chunk)
// Per-spinor occupation sums of one row, reduced from thread-private columns
// sacc[t * blockDim + thread]: spinor t by warp t mod (warps), lanes over the
// columns in a fixed order, then a shuffle tree; out[t] = the sum.
__device__ __forceinline__ void occ_rows_out(const double* sacc, int na, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5, nt = blockDim.x;
  for (int t = warp; t < na; t += nw) {
    double v = 0.0;
    for (int k = lane; k < nt; k += 32) v += sacc[t * nt + k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) out[t] = v;
  }
}

__global__ void k_hocc(const double* __restrict__ H, DevList Ls, int na, double* __restrict__ Hocc,
                       const int32_t* __restrict__ perm, int64_t ld) {
  __shared__ double sh[32];
  const int64_t r = blockIdx.x;
  double acc[64];
  for (int t = 0; t < na; ++t) acc[t] = 0.0;
  // perm: H in tile order ([r][slot], slot -> string perm[slot], -1 padding), row stride ld
  const int64_t ncol = perm ? ld : Ls.n;
  for (int64_t g = threadIdx.x; g < ncol; g += blockDim.x) {
    const int64_t a = perm ? (int64_t)perm[g] : g;
    if (a < 0) continue;
    const double h = H[r * ncol + g];
    for (uint64_t x = Ls.str[a]; x; x &= x - 1) acc[__ffsll((long long)x) - 1] += h;
  }
  for (int t = 0; t < na; ++t) {
    const double v = block_sum(acc[t], sh);
    if (threadIdx.x == 0) Hocc[r * na + t] = v;
  }
}

// Rows of every class with external spinors are tuples (h, p): a hole tuple h
// (none, one correlated core spinor, or a pair i<j) and a particle tuple p
// (likewise over correlated virtuals), row = h * n_p + p, pairs indexed
// b(b-1)/2 + a.  The marginals of per-row sums over the spinors a row
// contains are sums over tuples: for s a spinor of the tuple's set,
// out[b*ob + s*os + c*oc] (+)= sign * sum_{t contains s} in[(b*nt + t)*w + c]
// (arity 1: t = s; arity 2: t = pair(s,u) over u != s, in u order).
__global__ void k_tmarg(const double* __restrict__ in, int64_t nb, int64_t nt, int w, int arity, int ns, double sign,
                        int acc, double* __restrict__ out, int64_t ob, int64_t os, int64_t oc) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nb * ns * w) return;
  const int c = (int)(idx % w);
  const int64_t bs = idx / w;
  const int sp = (int)(bs % ns);
  const int64_t bb = bs / ns;
  const double* src = in + bb * nt * w + c;
  double v = 0.0;
  if (arity == 1) {
    v = src[(int64_t)sp * w];
  } else {
    for (int u = 0; u < ns; ++u) {
      if (u == sp) continue;
      const int64_t hi = max(sp, u), lo = min(sp, u);
      v += src[(hi * (hi - 1) / 2 + lo) * w];
    }
  }
  double* o = out + bb * ob + sp * os + c * oc;
  *o = acc ? *o + sign * v : sign * v;
}

// out[a*ldo + b] += in[pair(a,b)] for a != b (the pair entries of a tuple-set Gram matrix)
__global__ void k_pairplace(const double* __restrict__ in, int ns, double* __restrict__ out, int64_t ldo) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)ns * ns) return;
  const int a = (int)(idx / ns), b = (int)(idx % ns);
  if (a == b) return;
  const int64_t hi = max(a, b), lo = min(a, b);
  out[a * ldo + b] += in[hi * (hi - 1) / 2 + lo];
}

// out[h][c] = sum_p in[(h*np + p)*w + c]: one block per h, w <= 256; thread
// (q, c) sums p = q, q + nq, ... (coalesced over the flattened (p, c) index),
// then the nq partials of each c are added in q order
__global__ void k_midsum(const double* __restrict__ in, int64_t np, int w, double* __restrict__ out) {
  __shared__ double sh[256];
  const int nq = 256 / w, tid = threadIdx.x;
  const int c = tid % w, q = tid / w;
  const double* src = in + blockIdx.x * np * w;
  double v = 0.0;
  if (q < nq)
    for (int64_t p = q; p < np; p += nq) v += src[p * w + c];
  sh[tid] = v;
  __syncthreads();
  if (tid < w) {
    double t = 0.0;
    for (int k = 0; k < nq; ++k) t += sh[k * w + tid];
    out[blockIdx.x * (int64_t)w + tid] = t;
  }
}

// ------------------------------------------------------------------ reductions of the adjoint sums

// out[r] (+)= sum_c in[r*ncol + c] in index order
__global__ void k_rowsum(const double* __restrict__ in, int64_t nrow, int64_t ncol, int acc, double* __restrict__ out) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  double s = 0.0;
  for (int64_t c = 0; c < ncol; ++c) s += in[r * ncol + c];
  out[r] = acc ? out[r] + s : s;
}

// out[r] (+)= sum_c in[r*ncol + c] for long rows: one block per row, strided
// per-thread sums and a fixed-order block reduction
__global__ void k_rowsum_wide(const double* __restrict__ in, int64_t ncol, int acc, double* __restrict__ out) {
  __shared__ double sh[32];
  const int64_t r = blockIdx.x;
  double s = 0.0;
  for (int64_t c = threadIdx.x; c < ncol; c += blockDim.x) s += in[r * ncol + c];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[r] = acc ? out[r] + s : s;
}

// out[c] (+)= sum_r in[r*ncol + c] in index order
__global__ void k_colsum(const double* __restrict__ in, int64_t nrow, int64_t ncol, int acc, double* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  double s = 0.0;
  for (int64_t r = 0; r < nrow; ++r) s += in[r * ncol + c];
  out[c] = acc ? out[c] + s : s;
}

// scal_out[k] += sum_i in[2*i + k], k = 0, 1 (one block, fixed order)
__global__ void k_scalsum(const double* __restrict__ in, int64_t n, double* __restrict__ scal_out) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    a += in[2 * i];
    b += in[2 * i + 1];
  }
  a = block_sum(a, sh);
  b = block_sum(b, sh);
  if (threadIdx.x == 0) {
    scal_out[0] += a;
    scal_out[1] += b;
  }
}

// Nx[x] += sum over rows e whose particles / holes include x of hsum[e]
// (x indexes correlated core then correlated virtual spinors).
__global__ void k_xmarg(const RowInfo* __restrict__ rows, const double* __restrict__ hsum, int64_t M, int nx,
                        double* __restrict__ Nx) {
  __shared__ double sh[32];
  const int x = blockIdx.x;  // one block per external index
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < M; e += blockDim.x) {
    const RowInfo ri = rows[e];
    if (ri.s1 == x || ri.s2 == x || ri.i1 == x || ri.i2 == x) s += hsum[e];
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) Nx[x] += s;
}

// Nt[t] += sum_A hA[A] [t in A] over one string list (one block per t)
__global__ void k_amarg(DevList Ls, const double* __restrict__ hA, double* __restrict__ Nt) {
  __shared__ double sh[32];
  const int t = blockIdx.x;
  double s = 0.0;
  for (int64_t g = threadIdx.x; g < Ls.n; g += blockDim.x)
    if ((Ls.str[g] >> t) & 1) s += hA[g];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) Nt[t] += s;
}

// out[e] = sum_A conj(T[e][A]) d[A]  (one block per row)
__global__ void k_rowdot(const double2* __restrict__ T, const double2* __restrict__ d, int64_t N,
                         double2* __restrict__ out, const int32_t* __restrict__ perm, int64_t ld) {
  __shared__ double sh[32];
  const int64_t e = blockIdx.x;
  double2 acc = make_double2(0.0, 0.0);
  // perm: T in tile order (slot -> string perm[slot], -1 padding), row stride ld
  const int64_t ncol = perm ? ld : N;
  for (int64_t s = threadIdx.x; s < ncol; s += blockDim.x) {
    const int64_t A = perm ? (int64_t)perm[s] : s;
    if (A >= 0) acc = cfma(cconj(T[e * ncol + s]), d[A], acc);
  }
  const double re = block_sum(acc.x, sh), im = block_sum(acc.y, sh);
  if (threadIdx.x == 0) out[e] = make_double2(re, im);
}

// Gamma_f[a][i] += out[(i, a)] for the (1,1) rows e = i*nvc + a
__global__ void k_fock11(const double2* __restrict__ rowdot, DevSpace sp, double2* __restrict__ Gf) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)sp.ncc * sp.nvc) return;
  const int i = (int)(e / sp.nvc), a = (int)(e % sp.nvc);
  double2* dst = Gf + (int64_t)sp.vc[a] * sp.n_occ + sp.cc[i];
  dst->x += rowdot[e].x;
  dst->y += rowdot[e].y;
}

// ------------------------------------------------------------------ class (2,2)

// Per thread one string A; same tiling as the forward kernel.  Writes
//   cpart[yz][A] = sum_{ab in block} s (df/dv) |<ab||ij>|^2      (cbar_A = (2/n) c_A sum)
//   hpart[yz][A] = sum_{ab in block} s df/dD                     (string marginal)
//   vpart[cta][0..15] = per-virtual sums of s df/dD (a block, then b block), vpart[cta][16] = ij sum,
//   vpart[cta][17..18] = (sum s df/dD, sum s (df/dv) v)
__global__ void __launch_bounds__(256)
k_class22_bwd(DevList Ls, DevSpace sp, const double2* __restrict__ c, const double* __restrict__ g2,
              const double* __restrict__ epsh, const double* __restrict__ G, const double* __restrict__ E0p, double b,
              int nvb, double s, const double2* __restrict__ g1, double* __restrict__ cpart,
              double* __restrict__ hpart, double* __restrict__ vpart, double* __restrict__ part, int z0) {
  // core pair z0 + blockIdx.z; the chunk's partials are indexed by blockIdx.z
  const int zg = z0 + blockIdx.z;
  const double inv_n = 1.0 / g1[0].x;
  __shared__ double sGab[8][8], sG2[8][8], sAl[2][8];
  __shared__ double sh[32];
  int ba = 0, bb = 0;
  {
    int yb = blockIdx.y, k = 0;
    while (yb >= nvb - k) { yb -= nvb - k; ++k; }
    ba = k;
    bb = k + yb;
  }
  int iu, ju;
  pair_decode(zg, iu, ju);
  const int gi = sp.cc[iu], gj = sp.cc[ju];
  const int64_t nvp = pairs(sp.nvc);
  const int tid = threadIdx.x;
  if (tid < 64) {
    int x = tid >> 3, y = tid & 7;
    int a = ba * 8 + x, bq = bb * 8 + y;
    bool ok = a < sp.nvc && bq < sp.nvc && a < bq;
    sGab[x][y] = ok ? G[(int64_t)sp.vc[a] * sp.n + sp.vc[bq]] : 0.0;
    sG2[x][y] = ok ? g2[(int64_t)zg * nvp + pair_index(a, bq)] : 0.0;
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
  const int64_t A = blockIdx.x * (int64_t)blockDim.x + tid;
  double ha[8], hb[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) ha[k] = hb[k] = 0.0;
  double csum = 0.0, hsum = 0.0, gv = 0.0, acc = 0.0;
  if (A < Ls.n) {
    const double chi_ij = -epsh[gi] - epsh[gj] + G[(int64_t)gi * sp.n + gj];
    const double ct = *E0p - Ls.eA[A] + Ls.U[(int64_t)iu * Ls.n + A] + Ls.U[(int64_t)ju * Ls.n + A] - chi_ij;
    const double2 cv = c[A];
    const double c2 = (cv.x * cv.x + cv.y * cv.y) * inv_n;
    double inner = 0.0;  // sum w g(D): the forward's per-string sum, same order
    double pa[8], pb[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      int a = ba * 8 + k, bq = bb * 8 + k;
      pa[k] = (a < sp.nvc) ? sAl[0][k] + Ls.U[(int64_t)(sp.ncc + a) * Ls.n + A] : 0.0;
      pb[k] = (bq < sp.nvc) ? sAl[1][k] + Ls.U[(int64_t)(sp.ncc + bq) * Ls.n + A] : 0.0;
    }
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      const double cx = ct - pa[x];
#pragma unroll
      for (int y0 = 0; y0 < 8; y0 += 4) {  // the forward's groups of four denominators
        double Dv[4], q[4], rq[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          Dv[k] = cx - pb[y0 + k] - sGab[x][y0 + k];
          q[k] = sG2[x][y0 + k] != 0.0 ? en_q(Dv[k], b) : 1.0;
        }
        rcp4(q, rq);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int y = y0 + k;
          const double w = sG2[x][y];
          if (w == 0.0) continue;
          // df/dD is linear in v = w c2: accumulate it for v = w and scale
          // the sums by s c2 once per string
          double gk, hw;
          en_derivs_r(w, Dv[k], b, rq[k], gk, hw);
          hsum += hw;
          ha[x] += hw;
          hb[y] += hw;
          inner = fma(w, gk, inner);
        }
      }
    }
    acc = fma(cv.x, cv.x, cv.y * cv.y) * inner;
    const double sc2 = s * c2;
    csum = s * inner;   // sum s (df/dv) w
    gv = sc2 * inner;   // sum s (df/dv) v
    hsum *= sc2;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      ha[k] *= sc2;
      hb[k] *= sc2;
    }
  }
  const int64_t yz = (int64_t)blockIdx.z * gridDim.y + blockIdx.y;
  if (A < Ls.n) {
    cpart[yz * Ls.n + A] = csum;
    hpart[yz * Ls.n + A] = hsum;
  }
  const int64_t cta = yz * gridDim.x + blockIdx.x;
  {
    // the block's 18 sums at once: thread-private columns, then warp w sums
    // rows w, w + 8, w + 16 (lanes over the columns in a fixed order, a
    // shuffle tree)
    __shared__ double sv[18][256];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      sv[k][tid] = ha[k];
      sv[8 + k][tid] = hb[k];
    }
    sv[16][tid] = hsum;
    sv[17][tid] = gv;
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    for (int k = warp; k < 18; k += 8) {
      double v = 0.0;
      for (int q = lane; q < 256; q += 32) v += sv[k][q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) {
        if (k < 16) vpart[cta * 19 + k] = v;
        else if (k == 16) vpart[cta * 19 + 16] = vpart[cta * 19 + 17] = v;
        else vpart[cta * 19 + 18] = v;
      }
    }
  }
  if (part) {  // the forward's E2 partial of this block (global core-pair index)
    const double tot = block_sum(acc, sh);
    if (tid == 0) part[((int64_t)zg * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = tot;
  }
}

// Reduce the (2,2) per-CTA partials: Nx (virtual and core marginals), scalars.
__global__ void k_class22_marg(const double* __restrict__ vpart, int nx_blocks, int nvb, int64_t ncp, int z0,
                               DevSpace sp, double* __restrict__ Nx, double* __restrict__ scal) {
  // vpart holds core pairs z0 .. z0 + ncp - 1 (a chunk)
  // one block per correlated virtual a, per correlated core i, and one for
  // the two scalars; block-strided fixed-order sums
  __shared__ double sh[32];
  const int64_t nyb = (int64_t)nvb * (nvb + 1) / 2, nxb = nx_blocks;
  auto yidx = [&](int ba, int bb) { return (int64_t)ba * nvb - (int64_t)ba * (ba - 1) / 2 + (bb - ba); };
  const int x = blockIdx.x;
  double s = 0.0, s2 = 0.0;
  if (x < sp.nvc) {
    const int blk = x / 8, off = x % 8;
    const int64_t n = ncp * nvb * nxb;
    for (int64_t idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const int64_t z = idx / ((int64_t)nvb * nxb), xb = idx % nxb;
      const int m = (int)((idx / nxb) % nvb);   // the other virtual block of the pair
      if (m >= blk) s += vpart[((z * nyb + yidx(blk, m)) * nxb + xb) * 19 + off];
      if (m <= blk) s += vpart[((z * nyb + yidx(m, blk)) * nxb + xb) * 19 + 8 + off];
    }
  } else if (x < sp.nvc + sp.ncc) {
    const int i = x - sp.nvc;
    const int64_t per = nyb * nxb;
    for (int64_t idx = threadIdx.x; idx < ncp * per; idx += blockDim.x) {
      const int64_t z = idx / per;
      int iu, ju;
      pair_decode(z0 + z, iu, ju);
      if (iu == i || ju == i) s += vpart[idx * 19 + 16];
    }
  } else {
    for (int64_t k = threadIdx.x; k < ncp * nyb * nxb; k += blockDim.x) {
      s += vpart[k * 19 + 17];
      s2 += vpart[k * 19 + 18];
    }
  }
  s = block_sum(s, sh);
  s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    if (x < sp.nvc) Nx[sp.ncc + x] += s;
    else if (x < sp.nvc + sp.ncc) Nx[x - sp.nvc] += s;
    else {
      scal[0] += s;
      scal[1] += s2;
    }
  }
}

// ------------------------------------------------------------------ gather classes, pass 1

// Amplitudes and denominator weights of the gather classes, one thread per
// (row, string): T[row][A] = t_K, H[row][A] = s df/dD.  cls 1: (0,1) rows a;
// cls 3: (1,0) rows i; cls 0: (0,0) one row.
__global__ void k_gather_t(int cls, DevList Lx, DevList L12, DevList L02, DevList L21, DevList L11, DevDas das,
                           DevSpace sp, const int64_t* __restrict__ binom, const double2* __restrict__ DT,
                           const double2* __restrict__ DTU, const double2* __restrict__ DTD,
                           const double2* __restrict__ DTDU, const double2* __restrict__ X01,
                           const double2* __restrict__ X10, const double2* __restrict__ X00,
                           const double2* __restrict__ f, const double* __restrict__ epsh,
                           const double* __restrict__ E0p, double b, double s, const double2* __restrict__ g1,
                           double2* __restrict__ T, double* __restrict__ H, double* __restrict__ GV,
                           double* __restrict__ part) {
  __shared__ double sh[32];
  const double inv_n = 1.0 / g1[0].x, s2n = 2.0 * s * inv_n;
  const int row = blockIdx.y;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (g < Lx.n) {
  const uint64_t A = Lx.str[g];
  const int na = sp.n_act, ntp = (int)pairs(na);
  double2 V = make_double2(0.0, 0.0);
  double Dk = 0.0;  // denominators in the forward's operation order
  if (cls == 1) {
    const int ga = sp.vc[row];
    int64_t a12 = list_addr(L12, das, binom, A);
    if (a12 >= 0)
      for (int t = 0; t < na; ++t) V = cfma(f[(int64_t)ga * sp.n_occ + sp.a0 + t], DT[(int64_t)t * L12.n + a12], V);
    for (uint64_t x = A; x; x &= x - 1) {
      const int u = __ffsll((long long)x) - 1;
      const uint64_t B = A & ~(1ull << u);
      const int64_t a02 = list_addr(L02, das, binom, B);
      if (a02 < 0) continue;
      double2 sacc = make_double2(0.0, 0.0);
      const double2* Xr = X01 + ((int64_t)row * na + u) * ntp;
      for (int w = 1; w < na; ++w) {
        if ((B >> w) & 1) continue;
        for (int v = 0; v < w; ++v) {
          if ((B >> v) & 1) continue;
          const int vw = pair_index(v, w);
          sacc = cfma(Xr[vw], DTU[(int64_t)vw * L02.n + a02], sacc);
        }
      }
      if (popc_below(A, u) & 1) sacc = make_double2(-sacc.x, -sacc.y);
      V.x += sacc.x;
      V.y += sacc.y;
    }
    Dk = *E0p - Lx.eA[g] - epsh[ga] - Lx.U[(int64_t)(sp.ncc + row) * Lx.n + g];
  } else if (cls == 3) {
    const int gi = sp.cc[row];
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
        const double2* Xr = X10 + ((int64_t)row * pairs(na) + pair_index(t, u)) * na;
        double2 sacc = make_double2(0.0, 0.0);
        for (int v = 0; v < na; ++v) {
          if ((B >> v) & 1) continue;
          sacc = cfma(Xr[v], DT[(int64_t)v * L12.n + a12], sacc);
        }
        if ((popc_below(B, u) + popc_below(B, t)) & 1) sacc = make_double2(-sacc.x, -sacc.y);
        V.x += sacc.x;
        V.y += sacc.y;
      }
    }
    Dk = *E0p - Lx.eA[g] + epsh[gi] + Lx.U[(int64_t)row * Lx.n + g];
  } else {
    V = active_sigma(A, L11, L02, das, sp, binom, DTDU, DTU, X00, f);
    Dk = *E0p - Lx.eA[g];
  }
  const double v2 = fma(V.x, V.x, V.y * V.y);
  double gk, hk;
  en_derivs(v2 * inv_n, Dk, b, gk, hk);
  T[(int64_t)row * Lx.n + g] = make_double2(s2n * gk * V.x, s2n * gk * V.y);
  H[(int64_t)row * Lx.n + g] = s * hk;
  GV[(int64_t)row * Lx.n + g] = s * gk * v2 * inv_n;
  acc = v2 * gk;  // the forward's E2 term (gk = en_g(Dk, b))
  }
  if (part) {  // the forward's E2 partial of this block
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
}


// ------------------------------------------------------------------ gather classes, pass 2

// Gamma_f rows: out[r][k] = sum_A conj(T[r][A]) Dsrc(k, A) for the one-body
// part of a gather class (one block per (row, k)).
//   cls 1: Gamma_f[a][t]  += sum_A conj(T01[a][A]) D^t_A          (A in L01 -> L12 address)
//   cls 3: Gamma_f[t][i]  += sum_A conj(T10[i][A]) D^{t+}_A       (A in L10 -> L21 address)
//   cls 0: Gamma_f[t][u]  += sum_A conj(T00[A]) D^{t+u}_A         (A in L00 -> L11 address)
__global__ void k_gather_fock(int cls, DevList Lx, DevList Lsrc, DevDas das, DevSpace sp,
                              const int64_t* __restrict__ binom, const double2* __restrict__ Dsrc,
                              const double2* __restrict__ T, double2* __restrict__ Gf) {
  __shared__ double sh[32];
  const int na = sp.n_act;
  const int row = blockIdx.y, k = blockIdx.x;
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t g = threadIdx.x; g < Lx.n; g += blockDim.x) {
    const int64_t as = list_addr(Lsrc, das, binom, Lx.str[g]);
    if (as < 0) continue;
    const int64_t drow = (cls == 0) ? (1 + k) : k;
    acc = cfma(cconj(T[(int64_t)row * Lx.n + g]), Dsrc[drow * Lsrc.n + as], acc);
  }
  const double re = block_sum(acc.x, sh), im = block_sum(acc.y, sh);
  if (threadIdx.x == 0) {
    int64_t idx;
    if (cls == 1) idx = (int64_t)sp.vc[row] * sp.n_occ + sp.a0 + k;
    else if (cls == 3) idx = (int64_t)(sp.a0 + k) * sp.n_occ + sp.cc[row];
    else idx = (int64_t)(sp.a0 + k / na) * sp.n_occ + sp.a0 + k % na;
    Gf[idx].x += re;
    Gf[idx].y += im;
  }
}

// Gamma_D of the gather classes' one-body parts, one thread per string of the
// coupling table's list (sum over the class rows in order):
//   cls 1: Gamma_DT[t][A12]    += sum_a conj(T01[a][A]) f_at
//   cls 3: Gamma_DTD[t][A21]   += sum_i conj(T10[i][A]) f_ti
//   cls 0: Gamma_DTDU[1+tu][A11] += conj(T00[A]) f_tu
__global__ void k_gather_d1(int cls, DevList Lx, DevList Ltab, DevDas das, DevSpace sp, const int64_t* __restrict__ binom,
                            const double2* __restrict__ T, int nrow, const double2* __restrict__ f,
                            double2* __restrict__ GD) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= Ltab.n) return;
  const int64_t ax = list_addr(Lx, das, binom, Ltab.str[g]);
  if (ax < 0) return;
  const int na = sp.n_act;
  if (cls == 0) {
    const double2 tc = cconj(T[ax]);
    for (int t = 0; t < na; ++t)
      for (int u = 0; u < na; ++u) {
        double2* dst = GD + (int64_t)(1 + t * na + u) * Ltab.n + g;
        *dst = cfma(tc, f[(int64_t)(sp.a0 + t) * sp.n_occ + sp.a0 + u], *dst);
      }
    return;
  }
  for (int t = 0; t < na; ++t) {
    double2 acc = make_double2(0.0, 0.0);
    for (int r = 0; r < nrow; ++r) {
      const double2 fv = (cls == 1) ? f[(int64_t)sp.vc[r] * sp.n_occ + sp.a0 + t]
                                    : f[(int64_t)(sp.a0 + t) * sp.n_occ + sp.cc[r]];
      acc = cfma(cconj(T[(int64_t)r * Lx.n + ax]), fv, acc);
    }
    double2* dst = GD + (int64_t)t * Ltab.n + g;
    dst->x += acc.x;
    dst->y += acc.y;
  }
}

// Gamma_D of the gather classes' two-body parts, one thread per string B of
// the table's list, summing every (A, row) that reads D[x][B]:
//   cls 1: Gamma_DTU[vw][B]  += sum_{u not in B} sum_a conj(T01[a][B+u]) (-1)^{#(B+u)<u} <au||vw>
//   cls 3: Gamma_DT[v][B]    += sum_{t<u not in B} sum_i conj(T10[i][B+t+u]) s(B;t,u) <tu||iv>
//   cls 0: Gamma_DTU[vw][B]  += sum_{t<u not in B} conj(T00[B+t+u]) s(B;t,u) <tu||vw>
__global__ void k_gather_d2(int cls, DevList Lx, DevList Ltab, DevDas das, DevSpace sp, const int64_t* __restrict__ binom,
                            const double2* __restrict__ T, int nrow, const double2* __restrict__ X,
                            double2* __restrict__ GD) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= Ltab.n) return;
  const uint64_t B = Ltab.str[g];
  const int na = sp.n_act, ntp = (int)pairs(na);
  if (cls == 1) {
    for (int w = 1; w < na; ++w) {
      if ((B >> w) & 1) continue;
      for (int v = 0; v < w; ++v) {
        if ((B >> v) & 1) continue;
        const int vw = pair_index(v, w);
        double2 acc = make_double2(0.0, 0.0);
        for (int u = 0; u < na; ++u) {
          if ((B >> u) & 1) continue;
          const uint64_t A = B | (1ull << u);
          const int64_t ax = list_addr(Lx, das, binom, A);
          if (ax < 0) continue;
          double2 part = make_double2(0.0, 0.0);
          for (int a = 0; a < nrow; ++a)
            part = cfma(cconj(T[(int64_t)a * Lx.n + ax]), X[((int64_t)a * na + u) * ntp + vw], part);
          if (popc_below(A, u) & 1) part = make_double2(-part.x, -part.y);
          acc.x += part.x;
          acc.y += part.y;
        }
        double2* dst = GD + (int64_t)vw * Ltab.n + g;
        dst->x += acc.x;
        dst->y += acc.y;
      }
    }
    return;
  }
  const int nk = (cls == 3) ? na : ntp;
  for (int k = 0; k < nk; ++k) {
    if (cls == 3) {
      if ((B >> k) & 1) continue;
    } else {
      int v, w;
      pair_decode(k, v, w);
      if (((B >> v) & 1) || ((B >> w) & 1)) continue;
    }
    double2 acc = make_double2(0.0, 0.0);
    for (int u = 1; u < na; ++u) {
      if ((B >> u) & 1) continue;
      for (int t = 0; t < u; ++t) {
        if ((B >> t) & 1) continue;
        const uint64_t A = B | (1ull << t) | (1ull << u);
        const int64_t ax = list_addr(Lx, das, binom, A);
        if (ax < 0) continue;
        const int tu = pair_index(t, u);
        double2 part = make_double2(0.0, 0.0);
        if (cls == 3) {
          for (int i = 0; i < nrow; ++i)
            part = cfma(cconj(T[(int64_t)i * Lx.n + ax]), X[((int64_t)i * ntp + tu) * na + k], part);
        } else {
          part = cmul(cconj(T[ax]), X[(int64_t)tu * ntp + k]);
        }
        if ((popc_below(B, u) + popc_below(B, t)) & 1) part = make_double2(-part.x, -part.y);
        acc.x += part.x;
        acc.y += part.y;
      }
    }
    double2* dst = GD + (int64_t)k * Ltab.n + g;
    dst->x += acc.x;
    dst->y += acc.y;
  }
}

// ------------------------------------------------------------------ coupling tensors -> reference coefficients

// Gamma_c[L] = sum over every table entry D[x][A] = sign * c[L] of sign * Gamma_D[x][A],
// one thread per reference string L (the transpose of k_dtable).
__global__ void k_dscatter(int fam, DevList Ls, DevList Pl, DevDas das, const int64_t* __restrict__ binom,
                           const double2* __restrict__ GD, double2* __restrict__ Gc) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= Pl.n) return;
  const uint64_t L = Pl.str[l];
  const int na = das.n_act;
  double2 acc = make_double2(0.0, 0.0);
  auto add = [&](int64_t x, uint64_t A, int par) {
    const int64_t a = list_addr(Ls, das, binom, A);
    if (a < 0) return;
    double2 v = GD[x * Ls.n + a];
    if (par & 1) v = make_double2(-v.x, -v.y);
    acc.x += v.x;
    acc.y += v.y;
  };
  switch (fam) {
    case FAM_T:  // D^t_A = (-1)^{#A<t} c[A+t], t not in A: A = L - t
      for (int t = 0; t < na; ++t)
        if ((L >> t) & 1) add(t, L & ~(1ull << t), popc_below(L, t));
      break;
    case FAM_TD:  // D^{t+}_A = (-1)^{#A<t} c[A-t], t in A: A = L + t
      for (int t = 0; t < na; ++t)
        if (!((L >> t) & 1)) add(t, L | (1ull << t), popc_below(L, t));
      break;
    case FAM_TU:  // D^{tu}_A, A = L - t - u, parity #L<t + #(L-t)<u
      for (int u = 1; u < na; ++u)
        for (int t = 0; t < u; ++t)
          if (((L >> t) & 1) && ((L >> u) & 1))
            add(pair_index(t, u), L & ~(1ull << t) & ~(1ull << u),
                popc_below(L, t) + popc_below(L & ~(1ull << t), u));
      break;
    case FAM_TDUD:  // D^{t+u+}_A, A = L + t + u, parity #L<u + #L<t
      for (int u = 1; u < na; ++u)
        for (int t = 0; t < u; ++t)
          if (!((L >> t) & 1) && !((L >> u) & 1))
            add(pair_index(t, u), L | (1ull << t) | (1ull << u), popc_below(L, u) + popc_below(L, t));
      break;
    case FAM_TDU:  // row 0: A = L ; row 1+t*na+u: A = L - u + t (u in L; t == u or t not in L)
      add(0, L, 0);
      for (int u = 0; u < na; ++u) {
        if (!((L >> u) & 1)) continue;
        for (int t = 0; t < na; ++t) {
          if (t != u && ((L >> t) & 1)) continue;
          const uint64_t A = (L & ~(1ull << u)) | (1ull << t);
          add(1 + t * na + u, A, popc_below(L, u) + popc_below(A, t));
        }
      }
      break;
  }
  Gc[l].x += acc.x;
  Gc[l].y += acc.y;
}

// scal[0] += sum H, scal[1] += sum GV (one block, fixed order)
__global__ void k_sum2(const double* __restrict__ H, const double* __restrict__ GV, int64_t n, double* __restrict__ scal) {
  __shared__ double sh[32];
  double x = 0.0, y = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    x += H[i];
    y += GV[i];
  }
  x = block_sum(x, sh);
  y = block_sum(y, sh);
  if (threadIdx.x == 0) {
    scal[0] += x;
    scal[1] += y;
  }
}

// E0 term of the h coefficient: Gamma_f[t][u] += (sum eta / n) gamma_tu
__global__ void k_e0grad(const double2* __restrict__ g1, const double* __restrict__ scal, DevSpace sp,
                         double2* __restrict__ Gf) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int na = sp.n_act;
  if (k >= na * na) return;
  const double w = scal[0] / g1[0].x;
  const int t = k / na, u = k % na;
  double2* dst = Gf + (int64_t)(sp.a0 + t) * sp.n_occ + sp.a0 + u;
  dst->x += w * g1[1 + k].x;
  dst->y += w * g1[1 + k].y;
}

// Diagonal coefficient of h: correlated core +Nx, active -Nt, correlated virtual -Nx
__global__ void k_nd(DevSpace sp, const double* __restrict__ Nx, const double* __restrict__ Nt, double* __restrict__ Nd) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= sp.n) return;
  double v = 0.0;
  if (p >= sp.a0 && p < sp.v0) v = -Nt[p - sp.a0];
  for (int i = 0; i < sp.ncc; ++i)
    if (sp.cc[i] == p) v = Nx[i];
  for (int a = 0; a < sp.nvc; ++a)
    if (sp.vc[a] == p) v = -Nx[sp.ncc + a];
  Nd[p] = v;
}

// cbar = conj(Gamma_c) + (2/n) c (s * sum22 [per string, (2,2)])
//        + (2/n) eta (sigma' - E0' c) - (2/n) gv c
// scal = (sum eta, sum s (df/dv) v) over every class.
__global__ void k_cbar(int64_t np, const double2* __restrict__ Gc, const double* __restrict__ c22,
                       const double2* __restrict__ c, const double2* __restrict__ sigma, const double* __restrict__ scal,
                       const double* __restrict__ E0p, const double2* __restrict__ g1, double2* __restrict__ out) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= np) return;
  const double n = g1[0].x, two_n = 2.0 / n;
  const double eta = scal[0], gv = scal[1], e0p = *E0p;
  const double2 cv = c[l], sg = sigma[l];
  const double a = two_n * ((c22 ? c22[l] : 0.0) - gv);
  double2 v = cconj(Gc[l]);
  v.x += a * cv.x + two_n * eta * (sg.x - e0p * cv.x);
  v.y += a * cv.y + two_n * eta * (sg.y - e0p * cv.y);
  out[l] = v;
}

// hbar = Hermitian part of conj(Gamma_h), Gamma_h = Gamma_f (+ diagonal terms):
//   Gamma_h[p][p] += Nd[p] (denominators and E0)
__global__ void k_hbar(DevSpace sp, const double2* __restrict__ Gf, const double* __restrict__ Nd, double2* __restrict__ gh) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int n = sp.n;
  if (idx >= (int64_t)n * n) return;
  const int p = (int)(idx / n), q = (int)(idx % n);
  auto coef = [&](int x, int y) {
    double2 v = (y < sp.n_occ) ? Gf[(int64_t)x * sp.n_occ + y] : make_double2(0.0, 0.0);
    if (x == y) v.x += Nd[x];
    return v;
  };
  const double2 a = coef(p, q), bq = coef(q, p);
  // Hermitian projection of conj(Gamma): (conj(G_pq) + G_qp) / 2
  gh[idx] = make_double2(0.5 * (a.x + bq.x), 0.5 * (-a.y + bq.y));
}


// ------------------------------------------------------------------ factor gradient

// Pair-space coefficients of the chemists' integrals: pi = p * n_occ + y.
// Entry (row, col) of block `mode` with coefficient G (dE2 = Re G d<pq||rs>)
// adds G to (pr|qs) and -G to (ps|qr).  Within one launch every slot is
// written by one entry at most.
__global__ void k_gint(int mode, DevSpace sp, const double2* __restrict__ Gam, int64_t rows, int cols, int ld,
                       double2* __restrict__ Gt, int64_t npair) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= rows * (int64_t)cols) return;
  const int64_t row = idx / cols;
  const int col = (int)(idx % cols);
  int p, q, r, s;
  if (int_indices(mode, sp, row, col, p, q, r, s)) return;  // one-body column: handled by Gamma_f
  const double2 v = Gam[row * ld + col];
  const int no = sp.n_occ;
  double2* a = Gt + ((int64_t)p * no + r) * npair + (int64_t)q * no + s;
  double2* b = Gt + ((int64_t)p * no + s) * npair + (int64_t)q * no + r;
  a->x += v.x;
  a->y += v.y;
  b->x -= v.x;
  b->y -= v.y;
}

// Shifted amplitudes of a gather class for rows [row0, row0 + gridDim.y) and
// every shift z = blockIdx.z: one removed spinor t = z (pairs == 0) or a pair
// t < u with z = u(u-1)/2 + t.  Tsh[(y*S + z)*nB + g] = conj(T[row][A]) * sign
// for A = B_g + t (+ u), the sign of the coupling-table entry D_B the class
// reads for A; zero when t or u is in B or A is not in the class list.
__global__ void k_tshift(DevList Lx, DevList Ltab, DevDas das, const int64_t* __restrict__ binom,
                         const double2* __restrict__ T, int row0, int pairs_mode, double2* __restrict__ Tsh) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= Ltab.n) return;
  const int y = blockIdx.y, z = blockIdx.z, S = gridDim.z;
  int t = z, u = -1;
  if (pairs_mode) pair_decode(z, t, u);
  const uint64_t B = Ltab.str[g];
  double2 v = make_double2(0.0, 0.0);
  const bool clash = ((B >> t) & 1) || (u >= 0 && ((B >> u) & 1));
  if (!clash) {
    const uint64_t A = B | (1ull << t) | (u >= 0 ? (1ull << u) : 0ull);
    const int64_t ax = list_addr(Lx, das, binom, A);
    if (ax >= 0) {
      v = cconj(T[(int64_t)(row0 + y) * Lx.n + ax]);
      const int par = (u < 0) ? popc_below(A, t) : popc_below(B, u) + popc_below(B, t);
      if (par & 1) v = make_double2(-v.x, -v.y);
    }
  }
  Tsh[((int64_t)y * S + z) * Ltab.n + g] = v;
}

// Row-owner pass of class (2,2): one block per row (i<j, a<b).  For every A:
// eta = s df/dD and s (df/dv) |c_A|^2 / n; writes hsum[row], Hocc[row][t],
// P22[row] = sum_A s (df/dv) |c_A|^2 / n.
__global__ void __launch_bounds__(256)
k_class22_rows(DevList Ls, DevSpace sp, const double2* __restrict__ c, const double* __restrict__ g2,
               const double* __restrict__ epsh, const double* __restrict__ G, const double* __restrict__ E0p, double b,
               double s, const double2* __restrict__ g1, double* __restrict__ hsum, double* __restrict__ Hocc,
               double* __restrict__ P22) {
  __shared__ double sh[32];
  const int64_t nvp = pairs(sp.nvc);
  const int64_t row = blockIdx.x;
  int iu, ju, au, bu;
  pair_decode(row / nvp, iu, ju);
  pair_decode(row % nvp, au, bu);
  const int gi = sp.cc[iu], gj = sp.cc[ju], ga = sp.vc[au], gb = sp.vc[bu];
  const double w = g2[row];
  const double inv_n = 1.0 / g1[0].x;
  const double chi = -epsh[gi] - epsh[gj] + G[(int64_t)gi * sp.n + gj] + epsh[ga] + epsh[gb] + G[(int64_t)ga * sp.n + gb] -
                     G[(int64_t)gi * sp.n + ga] - G[(int64_t)gi * sp.n + gb] - G[(int64_t)gj * sp.n + ga] -
                     G[(int64_t)gj * sp.n + gb];
  const double e0p = *E0p;
  const int na = sp.n_act;
  extern __shared__ double sacc[];  // thread-private columns of the occupation sums
  const int nt = blockDim.x;
  double hs = 0.0, p22 = 0.0;
  for (int t = 0; t < na; ++t) sacc[t * nt + threadIdx.x] = 0.0;
  const double* Ua = Ls.U + (int64_t)(sp.ncc + au) * Ls.n;
  const double* Ub = Ls.U + (int64_t)(sp.ncc + bu) * Ls.n;
  const double* Ui = Ls.U + (int64_t)iu * Ls.n;
  const double* Uj = Ls.U + (int64_t)ju * Ls.n;
  // four strings per step (stride blockDim), their denominators inverted
  // together; df/dD is linear in v = w c2, so it is taken for v = w and scaled
  for (int64_t A0 = threadIdx.x; A0 < Ls.n; A0 += 4 * (int64_t)blockDim.x) {
    double Dv[4], q[4], rq[4], c2[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t A = A0 + k * (int64_t)blockDim.x;
      const bool ok = A < Ls.n;
      Dv[k] = ok ? e0p - Ls.eA[A] - chi - Ua[A] - Ub[A] + Ui[A] + Uj[A] : 1.0;
      q[k] = ok ? en_q(Dv[k], b) : 1.0;
      const double2 cv = ok ? c[A] : make_double2(0.0, 0.0);
      c2[k] = (cv.x * cv.x + cv.y * cv.y) * inv_n;
    }
    rcp4(q, rq);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t A = A0 + k * (int64_t)blockDim.x;
      if (A >= Ls.n) break;
      double gk, hw;
      en_derivs_r(w, Dv[k], b, rq[k], gk, hw);
      const double hk = c2[k] * hw;
      hs += hk;
      p22 = fma(gk, c2[k], p22);
      for (uint64_t x = Ls.str[A]; x; x &= x - 1) sacc[(__ffsll((long long)x) - 1) * nt + threadIdx.x] += hk;
    }
  }
  hs *= s;
  p22 *= s;
  for (int t = 0; t < na; ++t) sacc[t * nt + threadIdx.x] *= s;
  double v = block_sum(hs, sh);
  if (threadIdx.x == 0) hsum[row] = v;
  v = block_sum(p22, sh);  // (its barriers also order the column writes above)
  if (threadIdx.x == 0) P22[row] = v;
  occ_rows_out(sacc, na, Hocc + row * na);
}

// Gamma of <ab||ij>: 2 conj(g) P22
__global__ void k_g22coef(const double2* __restrict__ g, const double* __restrict__ P22, int64_t n,
                          double2* __restrict__ out) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  out[k] = make_double2(2.0 * P22[k] * g[k].x, -2.0 * P22[k] * g[k].y);
}

// Ntt[t][u] += sum_A hA[A] [t, u in A] (one block per ordered pair, t != u)
__global__ void k_ntt(DevList Ls, const double* __restrict__ hA, int na, double* __restrict__ Ntt) {
  __shared__ double sh[32];
  const int t = blockIdx.x / na, u = blockIdx.x % na;
  if (t == u) return;
  const uint64_t m = (1ull << t) | (1ull << u);
  double acc = 0.0;
  for (int64_t g = threadIdx.x; g < Ls.n; g += blockDim.x)
    if ((Ls.str[g] & m) == m) acc += hA[g];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) Ntt[t * na + u] += acc;
}

// Coefficient of G_pq (real, ordered entries):
//   eps^_p = h_pp + sum_{k in core} G_pk            -> Nd[p] on (p, k)
//   e_A    = ... + 1/2 sum_{t != u in A} G_tu         -> -1/2 Ntt[t][u]
//   chi_e  = ... + G of hole / particle pairs        -> -1/2 Ge[x][y]
//   U[x][A] = sum_{t in A} G_{X(x), t}              -> -Gea[x][t]
__global__ void k_gg(DevSpace sp, const double* __restrict__ Nd, const double* __restrict__ Ntt,
                     const double* __restrict__ Ge, const double* __restrict__ Gea, double* __restrict__ GG) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int n = sp.n, na = sp.n_act, nx = sp.nx;
  if (idx >= (int64_t)n * n) return;
  const int p = (int)(idx / n), q = (int)(idx % n);
  double v = 0.0;
  if (p != q) {
    if (q < sp.n_core) v += Nd[p];
    const bool pa = p >= sp.a0 && p < sp.v0, qa = q >= sp.a0 && q < sp.v0;
    if (pa && qa) v -= 0.5 * Ntt[(p - sp.a0) * na + (q - sp.a0)];
    int xp = -1, xq = -1;
    for (int i = 0; i < sp.ncc; ++i) {
      if (sp.cc[i] == p) xp = i;
      if (sp.cc[i] == q) xq = i;
    }
    for (int a = 0; a < sp.nvc; ++a) {
      if (sp.vc[a] == p) xp = sp.ncc + a;
      if (sp.vc[a] == q) xq = sp.ncc + a;
    }
    if (xp >= 0 && xq >= 0) v -= 0.5 * Ge[xp * nx + xq];
    if (xp >= 0 && qa) v -= Gea[xp * na + (q - sp.a0)];
  }
  GG[idx] = v;
}

// Gh = Gt + Gt^T (pair space)
__global__ void k_symm(const double2* __restrict__ Gt, int64_t npair, double2* __restrict__ Gh) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= npair * npair) return;
  const int64_t a = idx / npair, b = idx % npair;
  const double2 x = Gt[idx], y = Gt[b * npair + a];
  Gh[idx] = make_double2(x.x + y.x, x.y + y.y);
}

// Coefficient of dB^L_pq for every factor (complex, n x n per L):
//   integrals: w_L Cs[L][p*no + q] (q < n_occ), Cs = Bo Gh^T
//   G:         -w_L (GG_pq + GG_qp) B_qp (p != q); diagonal: w_L sum_r (GG_pr + GG_rp) B_rr
//   f:         w_L tr_L Gf[p][q] (q < n_occ); core k: diagonal w_L sum Gf B, and the
//              -w_L sum_y Gf[p][y] B_ky (q = k core) / -w_L sum_p' Gf[p'][q] B_p'p (p core) terms
__global__ void k_bcoef(DevSpace sp, const double2* __restrict__ Bc, const double2* __restrict__ Bx, int Lc, int Lx,
                        const double* __restrict__ wt, const double* __restrict__ dg, const double2* __restrict__ Cs,
                        const double* __restrict__ GG, const double2* __restrict__ Gf, const double2* __restrict__ ftr,
                        double2* __restrict__ GB) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int n = sp.n, no = sp.n_occ;
  if (idx >= (int64_t)(Lc + Lx) * n * n) return;
  const int L = (int)(idx / ((int64_t)n * n));
  const int64_t pq = idx % ((int64_t)n * n);
  const int p = (int)(pq / n), q = (int)(pq % n);
  const double2* B = (L < Lc) ? Bc + (int64_t)L * n * n : Bx + (int64_t)(L - Lc) * n * n;
  const double w = wt[L];
  double trc = 0.0;
  for (int k = 0; k < sp.n_core; ++k) trc += dg[(int64_t)L * n + k];
  double2 v = make_double2(0.0, 0.0);
  if (q < no) {
    const double2 cs = Cs[(int64_t)L * n * no + (int64_t)p * no + q];
    const double2 gf = Gf[(int64_t)p * no + q];
    v.x += w * (cs.x + trc * gf.x);
    v.y += w * (cs.y + trc * gf.y);
  }
  if (p != q) {
    const double gs = GG[(int64_t)p * n + q] + GG[(int64_t)q * n + p];
    const double2 bqp = B[(int64_t)q * n + p];
    v.x -= w * gs * bqp.x;
    v.y -= w * gs * bqp.y;
  } else {
    double acc = 0.0;
    for (int r = 0; r < n; ++r) acc += (GG[(int64_t)p * n + r] + GG[(int64_t)r * n + p]) * B[(int64_t)r * n + r].x;
    v.x += w * acc;
    if (p < sp.n_core) {
      v.x += w * ftr[L].x;
      v.y += w * ftr[L].y;
    }
  }
  if (q < sp.n_core) {  // -w sum_y Gf[p][y] B_qy
    double2 acc = make_double2(0.0, 0.0);
    for (int y = 0; y < no; ++y) acc = cfma(Gf[(int64_t)p * no + y], B[(int64_t)q * n + y], acc);
    v.x -= w * acc.x;
    v.y -= w * acc.y;
  }
  if (p < sp.n_core && q < no) {  // -w sum_p' Gf[p'][q] B_p'p
    double2 acc = make_double2(0.0, 0.0);
    for (int r = 0; r < n; ++r) acc = cfma(Gf[(int64_t)r * no + q], B[(int64_t)r * n + p], acc);
    v.x -= w * acc.x;
    v.y -= w * acc.y;
  }
  GB[idx] = v;
}

// ftr[L] = sum_{p, y < n_occ} Gf[p][y] B^L_py  (one block per factor)
__global__ void k_ftr(DevSpace sp, const double2* __restrict__ Bc, const double2* __restrict__ Bx, int Lc,
                      const double2* __restrict__ Gf, double2* __restrict__ ftr) {
  __shared__ double sh[32];
  const int L = blockIdx.x, n = sp.n, no = sp.n_occ;
  const double2* B = (L < Lc) ? Bc + (int64_t)L * n * n : Bx + (int64_t)(L - Lc) * n * n;
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t k = threadIdx.x; k < (int64_t)n * no; k += blockDim.x) {
    const int p = (int)(k / no), y = (int)(k % no);
    acc = cfma(Gf[k], B[(int64_t)p * n + y], acc);
  }
  const double re = block_sum(acc.x, sh), im = block_sum(acc.y, sh);
  if (threadIdx.x == 0) ftr[L] = make_double2(re, im);
}

// Weight gradient per factor: dE2/dw_L = 1/2 Re sum Bo Cs / w (integral part)
//   + sum GG (B_pp B_qq - |B_pq|^2) + Re sum_{p,y<no} Gf[p][y] (B_py tr - sum_k B_pk B_ky)
__global__ void k_gw(DevSpace sp, const double2* __restrict__ Bc, const double2* __restrict__ Bx, int Lc,
                     const double2* __restrict__ Bo, const double2* __restrict__ Cs, const double* __restrict__ GG,
                     const double2* __restrict__ Gf, const double* __restrict__ dg, double* __restrict__ gw) {
  __shared__ double sh[32];
  const int L = blockIdx.x, n = sp.n, no = sp.n_occ;
  const double2* B = (L < Lc) ? Bc + (int64_t)L * n * n : Bx + (int64_t)(L - Lc) * n * n;
  const int64_t np_ = (int64_t)n * no;
  double acc = 0.0;
  for (int64_t k = threadIdx.x; k < np_; k += blockDim.x) {
    const double2 a = Bo[(int64_t)L * np_ + k], c = Cs[(int64_t)L * np_ + k];
    acc += 0.5 * (a.x * c.x - a.y * c.y);
  }
  double trc = 0.0;
  for (int k = 0; k < sp.n_core; ++k) trc += dg[(int64_t)L * n + k];
  for (int64_t k = threadIdx.x; k < (int64_t)n * n; k += blockDim.x) {
    const int p = (int)(k / n), q = (int)(k % n);
    if (p != q) {
      const double2 bpq = B[k];
      acc += GG[k] * (dg[(int64_t)L * n + p] * dg[(int64_t)L * n + q] - (bpq.x * bpq.x + bpq.y * bpq.y));
    }
    if (q < no) {
      double2 t = make_double2(B[k].x * trc, B[k].y * trc);
      for (int kk = 0; kk < sp.n_core; ++kk) {
        const double2 m = cmul(B[(int64_t)p * n + kk], B[(int64_t)kk * n + q]);
        t.x -= m.x;
        t.y -= m.y;
      }
      const double2 gf = Gf[(int64_t)p * no + q];
      acc += gf.x * t.x - gf.y * t.y;
    }
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) gw[L] = acc;
}

// g_B = Hermitian projection of conj(coefficient), written per factor set
__global__ void k_bproj(int n, int Lc, int Lx, const double2* __restrict__ GB, double2* __restrict__ gBc,
                        double2* __restrict__ gBx) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)(Lc + Lx) * n * n) return;
  const int L = (int)(idx / ((int64_t)n * n));
  const int64_t pq = idx % ((int64_t)n * n);
  const int p = (int)(pq / n), q = (int)(pq % n);
  const double2 a = GB[idx], b = GB[(int64_t)L * n * n + (int64_t)q * n + p];
  const double2 v = make_double2(0.5 * (a.x + b.x), 0.5 * (-a.y + b.y));
  if (L < Lc) {
    if (gBc) gBc[idx] = v;
  } else if (gBx) {
    gBx[idx - (int64_t)Lc * n * n] = v;
  }
}

// E0 term of the <tu||vw> coefficient: GX00 += (sum eta / n) Gamma2
__global__ void k_x00e0(const double2* __restrict__ g1, const double2* __restrict__ g2, const double* __restrict__ scal,
                        int ntp, double2* __restrict__ GX00) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= (int64_t)ntp * ntp) return;
  const double w = scal[0] / g1[0].x;
  GX00[k].x += w * g2[k].x;
  GX00[k].y += w * g2[k].y;
}

// dE2/dlambda = sum over the extra set of w_x[L] dE2/dw_L
__global__ void k_dlambda(const double* __restrict__ gw, const double* __restrict__ wx, int Lc, int Lx,
                          double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int k = threadIdx.x; k < Lx; k += blockDim.x) acc += wx[k] * gw[Lc + k];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = acc;
}

}  // namespace e2
