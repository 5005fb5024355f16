// Dense-class contraction with FP64 accuracy on the bf16 tensor pipe.
//
// V[e,A] = sum_x W[e,x] D[x,A] (step a7) is formed from exact slices of its
// operands, as in Ozaki's error-free transformation of matrix products
// (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012): every row of W is
// scaled by a power of two 2^-sigma_e to magnitudes below 1 and cut into
// OZ_S slices of 8 significant bits, x = sum_i w_i 2^(-8 i), each w_i an
// integer of magnitude at most 256 (the first) or 128 (the others), chosen by
// rounding to nearest, so that the remainder after the last slice is below
// 2^(-8 OZ_S - 1).  Columns of D are cut the same way with 2^-tau_A.  The
// slices are exact in bf16, their products exact in FP32, and the sums of
// level 2 (i + j = 2) and level 3 (i + j = 3) are integers (after a fixed
// power-of-two scaling) below 2^24 as long as the real contraction length is
// at most 256: the FP32 tensor-core accumulation is then exact.  Level 4 has
// its own accumulator (integers times 2^-16, exact unless the slices are
// near their bounds throughout, and then rounded 2^-40 below the top level);
// levels 5 to OZ_S + 1 share one whose rounding is 2^-24 of a quantity
// already 2^-24 below the top.  The four accumulators are combined into a
// float-float value and scaled by 2^(sigma_e + tau_A).
//
// A complex product is one real product of twice the length:
//   [Wr | Wi] (M x 2K) times [[Dr, Di], [-Di, Dr]] (2K x 2N, columns of
//   each string interleaved re, im),
// so each thread's accumulator fragment holds Re V and Im V of one coupling.
//
// The Epstein-Nesbet epilogue (step a10) runs in float-float arithmetic on
// the FP32 pipe: D_K = E0' - chi_e - e_A - U[s1,A] - U[s2,A] + U[i1,A] +
// U[i2,A] from float-float copies of the per-string tables, g(D) = 1/D or
// the level-shifted D^3/(D^4 + b^2), and the tile's sum of |V|^2 g(D).
#include <cuda_bf16.h>

#include "e2_device.cuh"
#include "e2_df.cuh"
#include "e2_host.h"

namespace e2 {

namespace {

__device__ __forceinline__ double oz_block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) t += sh[i];
  return t;
}

// the slices of x (|x| < 1): w_i 2^(-8 (i - 1)), i = 1..OZ_S (each exact in bf16)
__device__ __forceinline__ void oz_cut(double x, float (&s)[OZ_S]) {
  double v = x;
#pragma unroll
  for (int i = 0; i < OZ_S; ++i) {
    const double t = v * 256.0;
    const double w = rint(t);
    s[i] = (float)w * __int_as_float((127 - 8 * i) << 23);  // w 2^(-8 i), exact
    v = t - w;                                               // exact
  }
}

// 2^k as a float, k clamped to the normal range
__device__ __forceinline__ float oz_pow2(int k) {
  k = max(-126, min(127, k));
  return __int_as_float((127 + k) << 23);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

}  // namespace

// ------------------------------------------------------------------ slicing

// Row slices of W (M x K complex, row stride ldw): A[s][row][k'] over the real
// length 2K ([Re | Im], zero to Kq), one exponent per row.  One warp per row;
// rows M..Mpad-1 are zero.
__global__ void k_oz_split_rows(const double2* __restrict__ W, int64_t M, int K, int64_t ldw, int Kq, int64_t Mpad,
                                __nv_bfloat16* __restrict__ A, int* __restrict__ rexp) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= Mpad) return;
  const double2* w = W + row * ldw;
  double m = 0.0;
  if (row < M)
    for (int k = lane; k < K; k += 32) m = fmax(m, fmax(fabs(w[k].x), fabs(w[k].y)));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  int e = 0;
  if (m > 0.0) frexp(m, &e);  // m < 2^e
  const double sc = ldexp(1.0, -e);
  for (int k = lane; k < Kq; k += 32) {
    double x = 0.0;
    if (row < M && k < 2 * K) x = (k < K ? w[k].x : w[k - K].y) * sc;
    float s[OZ_S];
    oz_cut(x, s);
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) A[((int64_t)i * Mpad + row) * Kq + k] = __float2bfloat16_rn(s[i]);
  }
  if (lane == 0) rexp[row] = e;
}

// Column slices of D (K x N complex, row-major): B[s][2A + h][k'] with
//   h = 0: (Dr[k], -Di[k]) over k' = k, K + k;  h = 1: (Di[k], Dr[k]),
// zero to Kq and for the padding strings N..Npad-1; one exponent per string.
// Block: 32 strings, 8 warps over k.
__global__ void k_oz_split_cols(const double2* __restrict__ D, int K, int64_t N, int Kq, int64_t Npad,
                                __nv_bfloat16* __restrict__ B, int* __restrict__ cexp) {
  __shared__ double sm[8][32];
  __shared__ int se[32];
  const int c = threadIdx.x & 31, kk = threadIdx.x >> 5;
  const int64_t col = (int64_t)blockIdx.x * 32 + c;
  const bool ok = col < N;
  double m = 0.0;
  if (ok)
    for (int k = kk; k < K; k += 8) {
      const double2 d = D[(int64_t)k * N + col];
      m = fmax(m, fmax(fabs(d.x), fabs(d.y)));
    }
  sm[kk][c] = m;
  __syncthreads();
  if (kk == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t = fmax(t, sm[i][c]);
    int e = 0;
    if (t > 0.0) frexp(t, &e);
    se[c] = e;
    if (col < Npad) cexp[col] = e;
  }
  __syncthreads();
  if (col >= Npad) return;
  const double sc = ldexp(1.0, -se[c]);
  const int64_t ps = 2 * Npad * (int64_t)Kq;  // one slice
  __nv_bfloat16* b0 = B + (2 * col) * (int64_t)Kq;
  __nv_bfloat16* b1 = b0 + Kq;
  for (int k = kk; k < K; k += 8) {
    const double2 d = ok ? D[(int64_t)k * N + col] : make_double2(0.0, 0.0);
    float sr[OZ_S], si[OZ_S];
    oz_cut(d.x * sc, sr);
    oz_cut(d.y * sc, si);
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) {
      b0[i * ps + k] = __float2bfloat16_rn(sr[i]);
      b0[i * ps + K + k] = __float2bfloat16_rn(-si[i]);
      b1[i * ps + k] = __float2bfloat16_rn(si[i]);
      b1[i * ps + K + k] = __float2bfloat16_rn(sr[i]);
    }
  }
  const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
  for (int k = 2 * K + kk; k < Kq; k += 8)
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) {
      b0[i * ps + k] = z;
      b1[i * ps + k] = z;
    }
}

// Float-float copies of e_A [n] and U [rows][n].
__global__ void k_oz_tables(const double* __restrict__ eA, const double* __restrict__ U, int64_t n, int64_t rows,
                            float2* __restrict__ eAdf, float2* __restrict__ Udf) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < rows * n) {
    const dfl u = df_from_double(U[idx]);
    Udf[idx] = make_float2(u.hi, u.lo);
  }
  if (idx < n) {
    const dfl a = df_from_double(eA[idx]);
    eAdf[idx] = make_float2(a.hi, a.lo);
  }
}

// ------------------------------------------------------------------ contraction + epilogue

// CTA tile: 64 rows x 64 strings (128 real columns), 8 warps of 32 rows x 16
// strings; real contraction staged in chunks of 32 (double-buffered with
// cp.async); per 16-step, the OZ_S (OZ_S + 1) / 2 slice pairs of levels up to
// OZ_S + 1 on mma.sync m16n8k16 bf16 with FP32 accumulators for levels 2, 3
// and 4 and one for the rest.
constexpr int OZ_BM = 64, OZ_BNR = 128, OZ_BK = 32, OZ_LD = OZ_BK + 8;
constexpr size_t OZ_STAGE = (size_t)OZ_S * (OZ_BM + OZ_BNR) * OZ_LD * 2;
constexpr size_t OZ_SMEM = 2 * OZ_STAGE;

__global__ void __launch_bounds__(256, 1)
k_class_oz(OzOperands op, int64_t M, int64_t N, const RowInfo* __restrict__ rows, const double* __restrict__ E0p,
           double b, double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char oz_smem[];
  __shared__ double sh[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3, g = lane >> 2, t = lane & 3;
  const int64_t m0 = (int64_t)blockIdx.x * OZ_BM, n0 = (int64_t)blockIdx.y * 64;
  const int Kq = op.Kq;
  auto sA = [&](int st, int s, int r, int k) {
    return (__nv_bfloat16*)(oz_smem + st * OZ_STAGE) + ((s * OZ_BM + r) * OZ_LD + k);
  };
  auto sB = [&](int st, int s, int r, int k) {
    return (__nv_bfloat16*)(oz_smem + st * OZ_STAGE) + (OZ_S * OZ_BM * OZ_LD + (s * OZ_BNR + r) * OZ_LD + k);
  };
  auto load = [&](int st, int kc) {
    const int k0 = kc * OZ_BK;
    for (int i = tid; i < OZ_S * OZ_BM * 4; i += 256) {
      const int s = i / (OZ_BM * 4), r = (i / 4) % OZ_BM, q = i & 3;
      cp_async16(sA(st, s, r, q * 8), op.A + ((int64_t)s * op.Mpad + m0 + r) * Kq + k0 + q * 8);
    }
    for (int i = tid; i < OZ_S * OZ_BNR * 4; i += 256) {
      const int s = i / (OZ_BNR * 4), r = (i / 4) % OZ_BNR, q = i & 3;
      cp_async16(sB(st, s, r, q * 8), op.B + ((int64_t)s * 2 * op.Npad + 2 * n0 + r) * Kq + k0 + q * 8);
    }
    cp_async_commit();
  };

  float acc[4][2][4][4];
#pragma unroll
  for (int l = 0; l < 4; ++l)
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < 4; ++ni)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[l][mi][ni][e] = 0.0f;

  const int nk = Kq / OZ_BK;
  load(0, 0);
  for (int kc = 0; kc < nk; ++kc) {
    const int st = kc & 1;
    if (kc + 1 < nk) {
      load(st ^ 1, kc + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < OZ_BK; ks += 16) {
      uint32_t bf[OZ_S][4][2];
#pragma unroll
      for (int s = 0; s < OZ_S; ++s)
#pragma unroll
        for (int np = 0; np < 2; ++np) {
          uint32_t r[4];
          ldsm_x4(r, sB(st, s, wn * 32 + np * 16 + (lane & 7) + (lane >> 4) * 8, ks + ((lane >> 3) & 1) * 8));
          bf[s][2 * np][0] = r[0];
          bf[s][2 * np][1] = r[1];
          bf[s][2 * np + 1][0] = r[2];
          bf[s][2 * np + 1][1] = r[3];
        }
#pragma unroll
      for (int sa = 0; sa < OZ_S; ++sa) {
        uint32_t af[2][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) ldsm_x4(af[mi], sA(st, sa, wm * 32 + mi * 16 + (lane & 15), ks + (lane >> 4) * 8));
#pragma unroll
        for (int sb = 0; sb < OZ_S - sa; ++sb) {
          const int l = sa + sb < 3 ? sa + sb : 3;
#pragma unroll
          for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) mma_bf16_16816(acc[l][mi][ni], af[mi], bf[sb][ni][0], bf[sb][ni][1]);
        }
      }
    }
    __syncthreads();
  }

  // epilogue, float-float: D_K = E0' - chi_e - e_A - U[s1,A] - U[s2,A] + U[i1,A] + U[i2,A]
  const double e0p = *E0p;
  const dfl bb = df_from_double(b * b);
  dfl sum{0.0f, 0.0f};
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int64_t row = m0 + wm * 32 + mi * 16 + g + hr * 8;
      if (row >= M) continue;
      const RowInfo ri = rows[row];
      const dfl base = df_from_double(e0p - ri.chi);
      const float2* U1 = op.Udf + (int64_t)ri.s1 * N;
      const float2* U2 = op.Udf + (int64_t)ri.s2 * N;
      const float2* U3 = op.Udf + (int64_t)ri.i1 * N;
      const float2* U4 = op.Udf + (int64_t)ri.i2 * N;
      const int er = op.rexp[row] - 16;
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int64_t col = n0 + wn * 16 + ni * 4 + t;
        if (col >= N) continue;
        const float sc = oz_pow2(er + op.cexp[col]);
        // levels 2 and 3 exactly (two_sum), then the small remainder
        const int cr = 2 * hr, ci = 2 * hr + 1;
        dfl vr = df_add_f(two_sum(acc[0][mi][ni][cr], acc[1][mi][ni][cr]),
                          __fadd_rn(acc[2][mi][ni][cr], acc[3][mi][ni][cr]));
        dfl vi = df_add_f(two_sum(acc[0][mi][ni][ci], acc[1][mi][ni][ci]),
                          __fadd_rn(acc[2][mi][ni][ci], acc[3][mi][ni][ci]));
        vr = df_scale(vr, sc);
        vi = df_scale(vi, sc);
        const dfl v2 = df_add(df_sqr(vr), df_sqr(vi));
        const float2 a = op.eAdf[col], u1 = U1[col], u2 = U2[col], u3 = U3[col], u4 = U4[col];
        dfl Dk = df_sub(base, dfl{a.x, a.y});
        Dk = df_sub(Dk, dfl{u1.x, u1.y});
        Dk = df_sub(Dk, dfl{u2.x, u2.y});
        Dk = df_add(Dk, dfl{u3.x, u3.y});
        Dk = df_add(Dk, dfl{u4.x, u4.y});
        dfl gk;
        if (b == 0.0) {
          gk = df_rcp(Dk);
        } else {  // level shift: g = D^3 / (D^4 + b^2)
          const dfl D2 = df_sqr(Dk);
          gk = df_mul(df_mul(Dk, D2), df_rcp(df_add(df_sqr(D2), bb)));
        }
        sum = df_add(sum, df_mul(v2, gk));
      }
    }
  const double tot = oz_block_sum(df_to_double(sum), sh);
  if (tid == 0 && partial) partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = tot;
}

// grid (Mpad / 64, Npad / 64); the shared-memory opt-in is set once per process
void launch_class_oz(cudaStream_t st, const OzOperands& op, int64_t M, int64_t N, const RowInfo* rows,
                     const double* E0p, double b, double* partial) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_class_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM);
    attr = true;
  }
  dim3 grid((unsigned)(op.Mpad / OZ_BM), (unsigned)(op.Npad / 64));
  (k_class_oz<<<grid, 256, OZ_SMEM, st>>>(op, M, N, rows, E0p, b, partial), ++g_launches);
}

}  // namespace e2
