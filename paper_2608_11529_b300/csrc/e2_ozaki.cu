// Dense-class contraction with FP64 accuracy on the bf16 tensor pipe.
//
// V[e,A] = sum_x W[e,x] D[x,A] (step a7) is formed from exact slices of its
// operands, as in Ozaki's error-free transformation of matrix products
// (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012): every row of W is
// scaled by a power of two 2^-sigma_e to magnitudes below 1 and cut into
// OZ_S slices of 8 significant bits, x = sum_i w_i 2^(-8 i), each w_i an
// integer of magnitude at most 256 (the first) or 128 (the others): x
// 2^(8 OZ_S) rounded to an integer, in balanced base-256 digits, so that the
// remainder after the last slice is at most 2^(-8 OZ_S - 1).  Columns of D
// are cut the same way with 2^-tau_A.  The
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

#include <mutex>

#include "e2_device.cuh"
#include "e2_df.cuh"
#include "e2_host.h"

namespace e2 {

// Once-per-device set-up (kernel attributes are per device): true on the
// first call for the current device, under a lock.
struct DeviceFlags {
  std::mutex mu;
  bool done[128] = {};
};
static bool first_use_on_device(DeviceFlags& f) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return true;
  std::lock_guard<std::mutex> lock(f.mu);
  if (f.done[dev]) return false;
  f.done[dev] = true;
  return true;
}
static DeviceFlags g_oz_attr;

namespace {

// The S slices of x relative to 2^e (|x| < 2^e), from the bit pattern of x in
// integer arithmetic (the FP64 pipe of this part is slow): N = x 2^(8 S - e)
// rounded to an integer (|N| <= 2^(8 S)), then balanced base-256 digits
// from the low end, d_i in [-128, 127] for i > 1 and d_1 in [-256, 256];
// slice i holds d_i 2^(-8 (i - 1)) (exact in bf16).  neg: slices of -x.
template <int S = OZ_S>
__device__ __forceinline__ void oz_digits(double x, int e, bool neg, float (&s)[S]) {
  long long bits = __double_as_longlong(x);
  if (neg) bits ^= (long long)0x8000000000000000ULL;
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long N = 0;
  if (ex != 0) {
    const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
    const int sh = 1075 + e - 8 * S - ex;  // at least 13 when |x| < 2^e
    if (sh < 63) N = (mant + (1LL << (sh - 1))) >> sh;
    if (bits < 0) N = -N;
  }
#pragma unroll
  for (int i = S - 1; i >= 1; --i) {
    const long long d = ((N + 128) & 255) - 128;
    s[i] = (float)(int)d * __int_as_float((127 - 8 * i) << 23);
    N = (N - d) >> 8;
  }
  s[0] = (float)(int)N;
}

// exponent e with |x| < 2^e from the largest magnitude's bit pattern (0 for 0)
__device__ __forceinline__ int oz_exp(unsigned long long maxbits) {
  const int ex = (int)(maxbits >> 52);
  if (ex >= 0x7FF) return OZ_NONFINITE;  // a NaN or an infinity in the row / column
  return ex ? ex - 1022 : 0;
}
__device__ __forceinline__ unsigned long long oz_mag(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFULL;
}

// f 2^(8 S - e) rounded to an integer, from the bits of a float (0 for 0)
template <int S>
__device__ __forceinline__ long long oz_fixed_f(float f, int e) {
  const int bits = __float_as_int(f);
  const int ex = (bits >> 23) & 0xFF;
  if (ex == 0) return 0;
  const long long mant = (bits & 0x7FFFFF) | 0x800000;
  const int sh = ex - 150 + 8 * S - e;  // left shift (at most 8 S - 23 when |f| < 2^e)
  long long N;
  if (sh >= 0) N = mant << sh;
  else if (sh > -40) N = (mant + (1LL << (-sh - 1))) >> (-sh);
  else N = 0;
  return bits < 0 ? -N : N;
}

// The S slices of a float-float value hi + lo relative to 2^e (|hi| < 2^e):
// N = round(hi 2^(8 S - e)) + round(lo 2^(8 S - e)), within one unit of
// rounding the sum, then the balanced digits as in oz_digits.
template <int S>
__device__ __forceinline__ void oz_digits_df(float hi, float lo, int e, bool neg, float (&s)[S]) {
  long long N = oz_fixed_f<S>(hi, e) + oz_fixed_f<S>(lo, e);
  if (neg) N = -N;
#pragma unroll
  for (int i = S - 1; i >= 1; --i) {
    const long long d = ((N + 128) & 255) - 128;
    s[i] = (float)(int)d * __int_as_float((127 - 8 * i) << 23);
    N = (N - d) >> 8;
  }
  s[0] = (float)(int)N;
}

// 2^k as a float, k clamped to the normal range; NaN for a scale that
// carries OZ_NONFINITE (a non-finite operand)
__device__ __forceinline__ float oz_pow2(int k) {
  if (k > OZ_NONFINITE / 2) return __int_as_float(0x7FC00000);
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

// Row slices of a complex M x K operand A (element (m, k) at A[m sam + k sak],
// conjugated if conj; FP64 pairs, or float-float quadruples when DF): out[s][m][k'] over the real length 2K ([Re | Im],
// zero to Kq), one exponent per row.  One warp per row; rows M..Mpad-1 are
// zero.
template <int S, bool DF>
__global__ void k_oz_slice_a(const void* __restrict__ Av, int64_t sam, int64_t sak, int conj, int64_t M, int K,
                             int Kq, int64_t Mpad, __nv_bfloat16* __restrict__ out, int* __restrict__ rexp) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= Mpad) return;
  // DF: the operand is float-float, (re.hi, re.lo, im.hi, im.lo) per element;
  // the row scale then comes from the high parts (|hi + lo| < 2^e whenever |hi| < 2^e)
  const double2* a = (const double2*)Av + row * sam;
  const float4* a4 = (const float4*)Av + row * sam;
  int e;
  if (DF) {
    unsigned m = 0;
    if (row < M)
      for (int k = lane; k < K; k += 32) {
        const float4 v = a4[k * sak];
        m = max(m, max((unsigned)__float_as_int(v.x) & 0x7FFFFFFFu, (unsigned)__float_as_int(v.z) & 0x7FFFFFFFu));
      }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int ex = (int)(m >> 23);
    e = ex >= 0xFF ? OZ_NONFINITE : ex ? ex - 126 : 0;
  } else {
    unsigned long long m = 0;
    if (row < M)
      for (int k = lane; k < K; k += 32) {
        const double2 v = a[k * sak];
        m = max(m, max(oz_mag(v.x), oz_mag(v.y)));
      }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    e = oz_exp(m);
  }
  auto cut = [&](int k, float (&sl)[S]) {
    if (row < M && k < 2 * K) {
      if (DF) {
        const float4 v = a4[(k < K ? k : k - K) * sak];
        if (k < K) oz_digits_df<S>(v.x, v.y, e, false, sl);
        else oz_digits_df<S>(v.z, v.w, e, conj != 0, sl);
      } else {
        if (k < K) oz_digits<S>(a[k * sak].x, e, false, sl);
        else oz_digits<S>(a[(k - K) * sak].y, e, conj != 0, sl);
      }
    } else {
#pragma unroll
      for (int i = 0; i < S; ++i) sl[i] = 0.0f;
    }
  };
  if ((K & 1) == 0) {
    // even K: each lane loads two complex elements k, k + 1 once and writes
    // the real halves at k, k + 1 and the imaginary halves at K + k, K + k + 1
    // (one 4-byte store per slice each)
    auto both = [&](int k, float (&re)[S], float (&im)[S]) {
      if (DF) {
        const float4 v = a4[k * sak];
        oz_digits_df<S>(v.x, v.y, e, false, re);
        oz_digits_df<S>(v.z, v.w, e, conj != 0, im);
      } else {
        const double2 v = a[k * sak];
        oz_digits<S>(v.x, e, false, re);
        oz_digits<S>(v.y, e, conj != 0, im);
      }
    };
    for (int k = 2 * lane; k < K; k += 64) {
      float r0[S], r1[S], i0[S], i1[S];
      if (row < M) {
        both(k, r0, i0);
        both(k + 1, r1, i1);
      } else {
#pragma unroll
        for (int i = 0; i < S; ++i) r0[i] = r1[i] = i0[i] = i1[i] = 0.0f;
      }
#pragma unroll
      for (int i = 0; i < S; ++i) {
        __nv_bfloat16* o = out + ((int64_t)i * Mpad + row) * Kq;
        *(__nv_bfloat162*)(o + k) = __floats2bfloat162_rn(r0[i], r1[i]);
        *(__nv_bfloat162*)(o + K + k) = __floats2bfloat162_rn(i0[i], i1[i]);
      }
    }
    const __nv_bfloat162 z2 = __floats2bfloat162_rn(0.0f, 0.0f);
    for (int k = 2 * K + 2 * lane; k < Kq; k += 64)
#pragma unroll
      for (int i = 0; i < S; ++i) *(__nv_bfloat162*)(out + ((int64_t)i * Mpad + row) * Kq + k) = z2;
  } else {
    for (int k = 2 * lane; k < Kq; k += 64) {  // two real k per lane: one 4-byte store per slice (Kq is even)
      float s0[S], s1[S];
      cut(k, s0);
      cut(k + 1, s1);
#pragma unroll
      for (int i = 0; i < S; ++i)
        *(__nv_bfloat162*)(out + ((int64_t)i * Mpad + row) * Kq + k) = __floats2bfloat162_rn(s0[i], s1[i]);
    }
  }
  if (lane == 0) rexp[row] = e;
}

// Largest magnitude (bit pattern) per column of a complex K x N operand B,
// over chunks of kchunk rows: grid (ceil(N / 32), ceil(K / kchunk)), atomicMax
// into cmax (zeroed by the caller; a maximum does not depend on the order).
__global__ void k_oz_colmax(const double2* __restrict__ B, int64_t sbk, int64_t sbn, int K, int64_t N, int kchunk,
                            unsigned long long* __restrict__ cmax) {
  __shared__ unsigned long long sm[8][32];
  const int c = threadIdx.x & 31, kk = threadIdx.x >> 5;
  const int64_t col = (int64_t)blockIdx.x * 32 + c;
  const int k0 = blockIdx.y * kchunk, k1 = min(K, k0 + kchunk);
  unsigned long long m = 0;
  if (col < N)
    for (int k = k0 + kk; k < k1; k += 8) {
      const double2 d = B[(int64_t)k * sbk + col * sbn];
      m = max(m, max(oz_mag(d.x), oz_mag(d.y)));
    }
  sm[kk][c] = m;
  __syncthreads();
  if (kk == 0 && col < N) {
    unsigned long long t = 0;
    for (int i = 0; i < 8; ++i) t = max(t, sm[i][c]);
    atomicMax(cmax + col, t);
  }
}

// Column slices of a complex K x N operand B (element (k, n) at B[k sbk +
// n sbn], conjugated if conj): out[s][2n + h][k'] with
//   h = 0: (Re B[k], -Im B[k]) over k' = k, K + k;  h = 1: (Im B[k], Re B[k]),
// zero to Kq and for the padding columns N..Npad-1; one exponent per column,
// from cmax (k_oz_colmax) or, when cmax is null, found by the block itself
// (then grid y must be 1).  Block: 32 columns x 8 warps over the rows
// [blockIdx.y kchunk, +kchunk).
template <int S>
__global__ void k_oz_slice_b(const double2* __restrict__ B, int64_t sbk, int64_t sbn, int conj, int K, int64_t N,
                             int Kq, int64_t Npad, __nv_bfloat16* __restrict__ out, int* __restrict__ cexp,
                             const unsigned long long* __restrict__ cmax, int kchunk) {
  __shared__ unsigned long long sm[8][32];
  __shared__ int se[32];
  const int c = threadIdx.x & 31, kk = threadIdx.x >> 5;
  const int64_t col = (int64_t)blockIdx.x * 32 + c;
  const bool ok = col < N;
  if (cmax) {
    if (kk == 0) se[c] = ok ? oz_exp(cmax[col]) : 0;
  } else {
    unsigned long long m = 0;
    if (ok)
      for (int k = kk; k < K; k += 8) {
        const double2 d = B[(int64_t)k * sbk + col * sbn];
        m = max(m, max(oz_mag(d.x), oz_mag(d.y)));
      }
    sm[kk][c] = m;
    __syncthreads();
    if (kk == 0) {
      unsigned long long t = 0;
      for (int i = 0; i < 8; ++i) t = max(t, sm[i][c]);
      se[c] = oz_exp(t);
    }
  }
  __syncthreads();
  if (col >= Npad) return;
  const int e = se[c];
  if (blockIdx.y == 0 && kk == 0) cexp[col] = e;
  const int64_t ps = 2 * Npad * (int64_t)Kq;  // one slice
  __nv_bfloat16* b0 = out + (2 * col) * (int64_t)Kq;
  __nv_bfloat16* b1 = b0 + Kq;
  const int k0 = blockIdx.y * kchunk, k1 = min(K, k0 + kchunk);
  for (int k = k0 + kk; k < k1; k += 8) {
    const double2 d = ok ? B[(int64_t)k * sbk + col * sbn] : make_double2(0.0, 0.0);
    float sr[S], sim[S];
    oz_digits<S>(d.x, e, false, sr);
    oz_digits<S>(d.y, e, conj != 0, sim);
#pragma unroll
    for (int i = 0; i < S; ++i) {
      b0[i * ps + k] = __float2bfloat16_rn(sr[i]);
      b0[i * ps + K + k] = __float2bfloat16_rn(-sim[i]);
      b1[i * ps + k] = __float2bfloat16_rn(sim[i]);
      b1[i * ps + K + k] = __float2bfloat16_rn(sr[i]);
    }
  }
  if (blockIdx.y == 0) {
    const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
    for (int k = 2 * K + kk; k < Kq; k += 8)
#pragma unroll
      for (int i = 0; i < S; ++i) {
        b0[i * ps + k] = z;
        b1[i * ps + k] = z;
      }
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
constexpr int OZ_VROW = 65;  // float4 stride of a staged row of V (65: no bank conflicts on the writes)
static_assert((size_t)OZ_VROW * 64 * 16 + 64 * 8 + 64 * 16 <= OZ_SMEM, "staged epilogue fits the stage buffers");

// Adjoint epilogue of one staged tile (rows m0.., strings n0..): per coupling
// f = |V|^2 g(D) / n (n = <c|c>) and, with s the seed,
//   t = s (2/n) g V                   -> adj.T (chunk-local rows; FP64, or float-float
//                                         quadruples when adj.t_df)
//   eta = s df/dD = s (|V|^2/n) g'(D)  -> adj.Hm (if set; float-float pairs)
// and the sums of eta over the tile's strings per row (adj.Hrow), over its
// rows per string (adj.Hcol), over the tile (scal[2 slot]), and of s f
// (scal[2 slot + 1]); all sums float-float in a fixed order.
struct OzSums {
  float hi, err;
  __device__ __forceinline__ void add(dfl x) {  // cascaded: hi parts by two_sum, the rest beside
    const dfl u = two_sum(hi, x.hi);
    hi = u.hi;
    err = __fadd_rn(err, __fadd_rn(u.lo, x.lo));
  }
  __device__ __forceinline__ dfl value() const { return fast_two_sum(hi, err); }
};

__device__ __forceinline__ dfl warp_df_sum(dfl v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = df_add(v, dfl{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
  return v;
}

template <int NS, int NH>
__device__ __forceinline__ void oz_adjoint_phase2(const OzOperands& op, int64_t M, int64_t N, int64_t m0, int64_t n0,
                                                  double b, const AdjOut& adj, const float4* sV, const float2* sBase,
                                                  const int4* sRI) {
  __shared__ float2 sCol[8][64];
  __shared__ float2 sTot[8][2];
  __shared__ float2 sC[3];  // 1/n, s, s 2/n (float-float)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    const double inv_n = 1.0 / adj.g1[0].x;
    const dfl a = df_from_double(inv_n), c = df_from_double(adj.s), d = df_from_double(2.0 * adj.s * inv_n);
    sC[0] = make_float2(a.hi, a.lo);
    sC[1] = make_float2(c.hi, c.lo);
    sC[2] = make_float2(d.hi, d.lo);
  }
  __syncthreads();
  const dfl inv_n{sC[0].x, sC[0].y}, sd{sC[1].x, sC[1].y}, s2n{sC[2].x, sC[2].y};
  const bool shifted = b != 0.0;
  const dfl bb = df_from_double(b * b), b3 = df_from_double(3.0 * b * b);
  const int64_t ct = gridDim.y;
  OzSums col[2] = {{0.f, 0.f}, {0.f, 0.f}}, ts{0.f, 0.f}, fs{0.f, 0.f};
  for (int rr = warp; rr < OZ_BM; rr += 8) {
    const int64_t row = m0 + rr;
    if (row >= M) break;
    const int4 ri = sRI[rr];
    const float2 bs = sBase[rr];
    OzSums rs{0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int cl = lane + 32 * h;
      const int64_t colg = n0 + cl;
      if (colg >= N) continue;
      const float4 v = sV[rr * OZ_VROW + cl];
      const dfl vr{v.x, v.y}, vi{v.z, v.w};
      const dfl p = two_prod(v.x, v.x), qq = two_prod(v.z, v.z);
      const dfl s2 = two_sum(p.hi, qq.hi);
      float e = __fadd_rn(__fadd_rn(p.lo, qq.lo), s2.lo);
      e = __fmaf_rn(__fadd_rn(v.x, v.x), v.y, e);
      e = __fmaf_rn(__fadd_rn(v.z, v.z), v.w, e);
      const dfl v2 = fast_two_sum(s2.hi, e);
      const float2 a = op.eAdf[colg];
      dfl Dk = df_sub(dfl{bs.x, bs.y}, dfl{a.x, a.y});
      if (NS >= 1) {
        const float2 u = op.Udf[(int64_t)ri.x * N + colg];
        Dk = df_sub(Dk, dfl{u.x, u.y});
      }
      if (NS >= 2) {
        const float2 u = op.Udf[(int64_t)ri.y * N + colg];
        Dk = df_sub(Dk, dfl{u.x, u.y});
      }
      if (NH >= 1) {
        const float2 u = op.Udf[(int64_t)ri.z * N + colg];
        Dk = df_add(Dk, dfl{u.x, u.y});
      }
      if (NH >= 2) {
        const float2 u = op.Udf[(int64_t)ri.w * N + colg];
        Dk = df_add(Dk, dfl{u.x, u.y});
      }
      const dfl vn = df_mul(v2, inv_n);  // |V|^2 / n
      dfl gk, hk;
      if (!shifted) {  // g = 1/D, dg/dD = -1/D^2
        gk = df_rcp(Dk);
        hk = df_mul(df_mul(vn, gk), gk);
        hk = dfl{-hk.hi, -hk.lo};
      } else {  // g = D^3 r, dg/dD = D^2 (3 b^2 - D^4) r^2, r = 1/(D^4 + b^2)
        const dfl D2 = df_sqr(Dk), D4 = df_sqr(D2);
        const dfl rq = df_rcp(df_add(D4, bb));
        gk = df_mul(df_mul(Dk, D2), rq);
        hk = df_mul(df_mul(df_mul(vn, D2), df_sub(b3, D4)), df_sqr(rq));
      }
      hk = df_mul(hk, sd);
      const dfl w = df_mul(s2n, gk);
      const int64_t o = (row - adj.m_base) * N + colg;
      const dfl tr = df_mul(w, vr), ti = df_mul(w, vi);
      if (adj.t_df)
        ((float4*)adj.T)[o] = make_float4(tr.hi, tr.lo, ti.hi, ti.lo);  // float-float, read by the row slicer
      else
        adj.T[o] = make_double2(df_to_double(tr), df_to_double(ti));
      if (adj.Hm) ((float2*)adj.Hm)[o] = make_float2(hk.hi, hk.lo);  // float-float, for k_hocc_df
      rs.add(hk);
      col[h].add(hk);
      ts.add(hk);
      fs.add(df_mul(v2, gk));
    }
    const dfl rsum = warp_df_sum(rs.value());  // the row's sum over the tile's strings
    if (lane == 0) adj.Hrow[(row - adj.m_base) * ct + blockIdx.y] = df_to_double(rsum);
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const dfl c = col[h].value();
    sCol[warp][lane + 32 * h] = make_float2(c.hi, c.lo);
  }
  const dfl t1 = warp_df_sum(ts.value()), t2 = warp_df_sum(fs.value());
  if (lane == 0) {
    sTot[warp][0] = make_float2(t1.hi, t1.lo);
    sTot[warp][1] = make_float2(t2.hi, t2.lo);
  }
  __syncthreads();
  if (tid < 64 && n0 + tid < N) {  // per string, over the 8 warps' rows in warp order
    dfl c{sCol[0][tid].x, sCol[0][tid].y};
    for (int w = 1; w < 8; ++w) c = df_add(c, dfl{sCol[w][tid].x, sCol[w][tid].y});
    adj.Hcol[(int64_t)blockIdx.x * N + n0 + tid] = df_to_double(c);
  }
  if (tid == 0) {
    dfl a{sTot[0][0].x, sTot[0][0].y}, f{sTot[0][1].x, sTot[0][1].y};
    for (int w = 1; w < 8; ++w) {
      a = df_add(a, dfl{sTot[w][0].x, sTot[w][0].y});
      f = df_add(f, dfl{sTot[w][1].x, sTot[w][1].y});
    }
    const int64_t slot = (int64_t)blockIdx.x * ct + blockIdx.y;
    adj.scal[2 * slot] = df_to_double(a);
    adj.scal[2 * slot + 1] = df_to_double(df_mul(df_mul(f, inv_n), sd));  // s f over the tile
  }
}

// NS, NH: the particles and holes of each row of the class (which U terms
// enter D), so that the epilogue is straight-line code.
// ADJ: the adjoint pass over the rows [adj.m_base, adj.m_base + adj.Mc) of a
// row chunk (grid x over the chunk's row tiles): amplitudes and sums of the
// FP64 kernel's adjoint mode (AdjOut), and no partial.
template <int NS, int NH, bool ADJ>
__global__ void __launch_bounds__(256, 1)
k_class_oz(OzOperands op, int64_t M, int64_t N, const RowInfo* __restrict__ rows, const double* __restrict__ E0p,
           double b, double* __restrict__ partial, AdjOut adj, unsigned long long* dmin) {
  extern __shared__ __align__(16) unsigned char oz_smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3, g = lane >> 2, t = lane & 3;
  // rows from adj.m_base: the adjoint's chunk, or in the forward the first row
  // tile of a shard (0 for all rows)
  const int64_t m0 = adj.m_base + (int64_t)blockIdx.x * OZ_BM, n0 = (int64_t)blockIdx.y * 64;
  if (ADJ) M = min(M, adj.m_base + adj.Mc);  // the chunk's last row
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

  // Epilogue, phase 1: the four levels of each coupling combined into
  // float-float Re V, Im V (scaled by 2^(sigma_e + tau_A)) and staged in the
  // free stage buffers, [64 rows][65] float4; the rows' E0' - chi_e and
  // spinor indices beside them (the only FP64 work of the kernel: 64 rows).
  float4* sV = (float4*)oz_smem;
  float2* sBase = (float2*)(oz_smem + OZ_VROW * 64 * 16);
  int4* sRI = (int4*)(oz_smem + OZ_VROW * 64 * 16 + 64 * 8);
  if (tid < 64) {
    const int64_t row = m0 + tid;
    float2 bs = make_float2(0.f, 0.f);
    int4 r4 = make_int4(0, 0, 0, 0);
    if (row < M) {
      const RowInfo ri = rows[row];
      const dfl d = df_from_double(*E0p - ri.chi);
      bs = make_float2(d.hi, d.lo);
      r4 = make_int4(ri.s1, ri.s2, ri.i1, ri.i2);
    }
    sBase[tid] = bs;
    sRI[tid] = r4;
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int rl = wm * 32 + mi * 16 + g + hr * 8;
      const int er = op.rexp[m0 + rl] - 16;  // rows to Mpad carry exponents
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int cl = wn * 16 + ni * 4 + t;
        const float sc = oz_pow2(er + op.cexp[n0 + cl]);
        const int cr = 2 * hr, ci = 2 * hr + 1;
        // levels 2 and 3 exactly (two_sum), the small remainder into the low part
        dfl vr = two_sum(acc[0][mi][ni][cr], acc[1][mi][ni][cr]);
        vr = fast_two_sum(vr.hi, __fadd_rn(vr.lo, __fadd_rn(acc[2][mi][ni][cr], acc[3][mi][ni][cr])));
        dfl vi = two_sum(acc[0][mi][ni][ci], acc[1][mi][ni][ci]);
        vi = fast_two_sum(vi.hi, __fadd_rn(vi.lo, __fadd_rn(acc[2][mi][ni][ci], acc[3][mi][ni][ci])));
        sV[rl * OZ_VROW + cl] = make_float4(__fmul_rn(vr.hi, sc), __fmul_rn(vr.lo, sc), __fmul_rn(vi.hi, sc),
                                            __fmul_rn(vi.lo, sc));
      }
    }
  __syncthreads();

  if constexpr (ADJ) {
    oz_adjoint_phase2<NS, NH>(op, M, N, m0, n0, b, adj, sV, sBase, sRI);
    return;
  }
  // Phase 2: one warp per row, lanes over the tile's strings (coalesced reads
  // of the float-float tables), four rows at a time so that each thread has
  // eight independent couplings in flight; eight partial sums, added in a
  // fixed order at the end.
  //   D_K = E0' - chi_e - e_A - U[s1,A] - U[s2,A] + U[i1,A] + U[i2,A]
  const bool shifted = b != 0.0;
  const dfl bb = df_from_double(b * b);  // once per thread
  float shi[8], serr[8];  // per slot: hi parts by two_sum, their errors beside
  unsigned dmk = 0xFFFFFFFFu;  // smallest |D| (high part) key of the thread
#pragma unroll
  for (int k = 0; k < 8; ++k) shi[k] = serr[k] = 0.0f;
#pragma unroll
  for (int rb = 0; rb < 8; rb += 4) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int rr = warp + 8 * (rb + q);
      const bool rok = m0 + rr < M;
      const int4 ri = sRI[rr];
      const float2 bs = sBase[rr];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int slot = q * 2 + h;
        const int cl = lane + 32 * h;
        const int64_t col = n0 + cl;
        if (!rok || col >= N) continue;
        const float4 v = sV[rr * OZ_VROW + cl];
        // |V|^2 = vr^2 + vi^2 from the exact squares of the high parts
        const dfl p = two_prod(v.x, v.x), qq = two_prod(v.z, v.z);
        const dfl s2 = two_sum(p.hi, qq.hi);
        float e = __fadd_rn(__fadd_rn(p.lo, qq.lo), s2.lo);
        e = __fmaf_rn(__fadd_rn(v.x, v.x), v.y, e);
        e = __fmaf_rn(__fadd_rn(v.z, v.z), v.w, e);
        const dfl v2 = fast_two_sum(s2.hi, e);
        const float2 a = op.eAdf[col];
        dfl Dk = df_sub(dfl{bs.x, bs.y}, dfl{a.x, a.y});
        if (NS >= 1) {
          const float2 u = op.Udf[(int64_t)ri.x * N + col];
          Dk = df_sub(Dk, dfl{u.x, u.y});
        }
        if (NS >= 2) {
          const float2 u = op.Udf[(int64_t)ri.y * N + col];
          Dk = df_sub(Dk, dfl{u.x, u.y});
        }
        if (NH >= 1) {
          const float2 u = op.Udf[(int64_t)ri.z * N + col];
          Dk = df_add(Dk, dfl{u.x, u.y});
        }
        if (NH >= 2) {
          const float2 u = op.Udf[(int64_t)ri.w * N + col];
          Dk = df_add(Dk, dfl{u.x, u.y});
        }
        if (bs.x < 1e7f) dmk = min(dmk, fkey(Dk.hi));  // rows outside Q sit at E0' - chi = 1e8
        dfl gk;
        if (!shifted) {
          gk = df_rcp(Dk);
        } else {  // level shift: g = D^3 / (D^4 + b^2)
          const dfl D2 = df_sqr(Dk);
          gk = df_mul(df_mul(Dk, D2), df_rcp(df_add(df_sqr(D2), bb)));
        }
        const dfl term = df_mul(v2, gk);
        const dfl u = two_sum(shi[slot], term.hi);
        shi[slot] = u.hi;
        serr[slot] = __fadd_rn(serr[slot], __fadd_rn(u.lo, term.lo));
      }
    }
  }
  dmin_flush_f(dmin, dmk);
  dfl tsum = fast_two_sum(shi[0], serr[0]);
#pragma unroll
  for (int k = 1; k < 8; ++k) tsum = df_add(tsum, fast_two_sum(shi[k], serr[k]));
  // block sum in float-float (fixed order: warp tree, then warps 0..7), one
  // conversion to double per CTA
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const dfl other{__shfl_xor_sync(0xffffffffu, tsum.hi, o), __shfl_xor_sync(0xffffffffu, tsum.lo, o)};
    tsum = df_add(tsum, other);
  }
  __shared__ float2 sW[8];
  if (lane == 0) sW[warp] = make_float2(tsum.hi, tsum.lo);
  __syncthreads();
  if (tid == 0 && partial) {
    dfl tot{sW[0].x, sW[0].y};
    for (int w = 1; w < 8; ++w) tot = df_add(tot, dfl{sW[w].x, sW[w].y});
    partial[(int64_t)blockIdx.y * adj.rt + adj.m_base / OZ_BM + blockIdx.x] = df_to_double(tot);
  }
}

// Forward: grid (Mpad / 64, Npad / 64).  Adjoint: grid (row tiles of the
// chunk, Npad / 64).  The shared-memory opt-in is set once per process.
template <bool ADJ>
static void set_oz_attr() {
  cudaFuncSetAttribute(k_class_oz<2, 0, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM);
  cudaFuncSetAttribute(k_class_oz<2, 1, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM);
  cudaFuncSetAttribute(k_class_oz<1, 2, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM);
  cudaFuncSetAttribute(k_class_oz<0, 2, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM);
}

static void launch_class_oz_mode(cudaStream_t st, int cls, const OzOperands& op, int64_t M, int64_t N,
                                 const RowInfo* rows, const double* E0p, double b, double* partial,
                                 const AdjOut* adj, unsigned long long* dmin, int64_t tm0, int64_t ntm) {
  // the attribute belongs to the device: set it on each device's first launch
  if (first_use_on_device(g_oz_attr)) {
    set_oz_attr<false>();
    set_oz_attr<true>();
  }
  AdjOut a = adj ? *adj : AdjOut{};
  if (!adj) {  // forward: row tiles tm0 .. tm0 + ntm - 1 of Mpad / 64, one partial slot each
    a.m_base = tm0 * OZ_BM;
    a.rt = op.Mpad / OZ_BM;
  }
  dim3 grid((unsigned)(adj ? (adj->Mc + OZ_BM - 1) / OZ_BM : ntm), (unsigned)(op.Npad / 64));
#define E2_OZ_LAUNCH(NS_, NH_)                                                                                   \
  if (adj)                                                                                                     \
    (k_class_oz<NS_, NH_, true><<<grid, 256, OZ_SMEM, st>>>(op, M, N, rows, E0p, b, nullptr, a, nullptr),      \
     ++g_launches);                                                                                            \
  else                                                                                                         \
    (k_class_oz<NS_, NH_, false><<<grid, 256, OZ_SMEM, st>>>(op, M, N, rows, E0p, b, partial, a, dmin),         \
     ++g_launches);
  switch (cls) {  // particles and holes of the rows
    case 2: E2_OZ_LAUNCH(2, 0) break;
    case 5: E2_OZ_LAUNCH(2, 1) break;
    case 7: E2_OZ_LAUNCH(1, 2) break;
    case 6: E2_OZ_LAUNCH(0, 2) break;
    default: break;
  }
#undef E2_OZ_LAUNCH
}

void launch_class_oz(cudaStream_t st, int cls, const OzOperands& op, int64_t M, int64_t N, const RowInfo* rows,
                     const double* E0p, double b, double* partial, unsigned long long* dmin, int64_t tm0,
                     int64_t ntm) {
  if (ntm < 0) ntm = op.Mpad / OZ_BM - tm0;
  if (ntm <= 0) return;
  launch_class_oz_mode(st, cls, op, M, N, rows, E0p, b, partial, nullptr, dmin, tm0, ntm);
}

void launch_class_oz_adj(cudaStream_t st, int cls, const OzOperands& op, int64_t M, int64_t N, const RowInfo* rows,
                         const double* E0p, double b, const AdjOut& adj) {
  launch_class_oz_mode(st, cls, op, M, N, rows, E0p, b, nullptr, &adj, nullptr, 0, 0);
}

// ------------------------------------------------------------------ general product

// C (+)= A B for complex FP64 operands through their slices (k_oz_slice_a/b):
// CTA tile 64 rows x 32 complex columns (64 real), 8 warps of 32 x 16 real;
// the four level accumulators of each output are exact over 256 real k and
// are flushed after every 256 into a float-float accumulator (so any
// contraction length keeps the per-256 exactness), which is scaled by
// 2^(rexp + cexp - 16) and written in FP64 at the end.  With lower >= 0 only
// tiles holding some column n <= lower + m are computed (a triangle).
struct OzGemm {
  const __nv_bfloat16* A;
  int64_t Mpad;
  const int* rexp;
  const __nv_bfloat16* B;
  int64_t Npad;
  const int* cexp;
  int Kq;
  int64_t M, N;
  double2* C;
  int64_t csm, csn;
  int beta;
  int64_t lower;
};

constexpr int OG_BM = 64, OG_BNR = 64, OG_BK = 32, OG_LD = OG_BK + 8;

template <int S>
__global__ void __launch_bounds__(256, 2) k_zgemm_sl(OzGemm q) {
  constexpr size_t og_stage = (size_t)S * (OG_BM + OG_BNR) * OG_LD * 2;
  extern __shared__ __align__(16) unsigned char og_smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3, g = lane >> 2, t = lane & 3;
  const int64_t m0 = (int64_t)blockIdx.x * OG_BM, n0 = (int64_t)blockIdx.y * (OG_BNR / 2);
  if (q.lower >= 0 && n0 > q.lower + m0 + OG_BM - 1) return;
  const int Kq = q.Kq;
  auto sA = [&](int st, int s, int r, int k) {
    return (__nv_bfloat16*)(og_smem + st * og_stage) + ((s * OG_BM + r) * OG_LD + k);
  };
  auto sB = [&](int st, int s, int r, int k) {
    return (__nv_bfloat16*)(og_smem + st * og_stage) + (S * OG_BM * OG_LD + (s * OG_BNR + r) * OG_LD + k);
  };
  auto load = [&](int st, int kc) {
    const int k0 = kc * OG_BK;
    for (int i = tid; i < S * OG_BM * 4; i += 256) {
      const int s = i / (OG_BM * 4), r = (i / 4) % OG_BM, c = i & 3;
      cp_async16(sA(st, s, r, c * 8), q.A + ((int64_t)s * q.Mpad + m0 + r) * Kq + k0 + c * 8);
    }
    for (int i = tid; i < S * OG_BNR * 4; i += 256) {
      const int s = i / (OG_BNR * 4), r = (i / 4) % OG_BNR, c = i & 3;
      cp_async16(sB(st, s, r, c * 8), q.B + ((int64_t)s * 2 * q.Npad + 2 * n0 + r) * Kq + k0 + c * 8);
    }
    cp_async_commit();
  };
  float acc[4][2][2][4];
  float dh[2][2][4], dl[2][2][4];  // float-float sums of the flushed 256-chunks
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        dh[mi][ni][e] = dl[mi][ni][e] = 0.0f;
#pragma unroll
        for (int l = 0; l < 4; ++l) acc[l][mi][ni][e] = 0.0f;
      }
  auto flush = [&]() {
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < 2; ++ni)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          dfl v = two_sum(acc[0][mi][ni][e], acc[1][mi][ni][e]);
          v = fast_two_sum(v.hi, __fadd_rn(v.lo, __fadd_rn(acc[2][mi][ni][e], acc[3][mi][ni][e])));
          const dfl d = df_add(dfl{dh[mi][ni][e], dl[mi][ni][e]}, v);
          dh[mi][ni][e] = d.hi;
          dl[mi][ni][e] = d.lo;
#pragma unroll
          for (int l = 0; l < 4; ++l) acc[l][mi][ni][e] = 0.0f;
        }
  };

  const int nk = Kq / OG_BK;
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
    for (int ks = 0; ks < OG_BK; ks += 16) {
      uint32_t bf[S][2][2];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        uint32_t r[4];
        ldsm_x4(r, sB(st, s, wn * 16 + (lane & 7) + (lane >> 4) * 8, ks + ((lane >> 3) & 1) * 8));
        bf[s][0][0] = r[0];
        bf[s][0][1] = r[1];
        bf[s][1][0] = r[2];
        bf[s][1][1] = r[3];
      }
#pragma unroll
      for (int sa = 0; sa < S; ++sa) {
        uint32_t af[2][4];
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) ldsm_x4(af[mi], sA(st, sa, wm * 32 + mi * 16 + (lane & 15), ks + (lane >> 4) * 8));
#pragma unroll
        for (int sb = 0; sb < S - sa; ++sb) {
          const int l = sa + sb < 3 ? sa + sb : 3;
#pragma unroll
          for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 2; ++ni) mma_bf16_16816(acc[l][mi][ni], af[mi], bf[sb][ni][0], bf[sb][ni][1]);
        }
      }
    }
    __syncthreads();
    if ((kc & 7) == 7 || kc + 1 == nk) flush();  // every 256 real k
  }
  // C[m][n] (+)= 2^(rexp + cexp - 16) (re, im)
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int64_t row = m0 + wm * 32 + mi * 16 + g + hr * 8;
      if (row >= q.M) continue;
      const int er = q.rexp[row] - 16;
#pragma unroll
      for (int ni = 0; ni < 2; ++ni) {
        const int64_t col = n0 + wn * 8 + ni * 4 + t;
        if (col >= q.N) continue;
        const int ek = er + q.cexp[col];
        const double sc = ek > OZ_NONFINITE / 2 ? __longlong_as_double(0x7FF8000000000000LL) : ldexp(1.0, ek);
        const double re = df_to_double(dfl{dh[mi][ni][2 * hr], dl[mi][ni][2 * hr]}) * sc;
        const double im = df_to_double(dfl{dh[mi][ni][2 * hr + 1], dl[mi][ni][2 * hr + 1]}) * sc;
        double2* c = q.C + row * q.csm + col * q.csn;
        if (q.beta) {
          const double2 o = *c;
          *c = make_double2(o.x + re, o.y + im);
        } else {
          *c = make_double2(re, im);
        }
      }
    }
}

size_t zgemm_sliced_bytes(int64_t M, int64_t N, int64_t K, int slices) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const int64_t Mpad = (M + OG_BM - 1) / OG_BM * OG_BM, Npad = (N + 31) / 32 * 32;
  const int64_t Kq = (2 * K + 31) / 32 * 32;
  return al((size_t)2 * slices * Mpad * Kq) + al(4 * (size_t)Mpad) + al((size_t)2 * slices * 2 * Npad * Kq) +
         al(4 * (size_t)Npad) + al(8 * (size_t)Npad);
}

// the column slicer's rows per block: all of them for a short contraction,
// chunks of 256 (after a column-maximum pass) for a long one
static constexpr int OZ_KCHUNK = 256;

template <int S>
static void zgemm_sliced_run(cudaStream_t st, int64_t M, int64_t N, int64_t Nb, int64_t K, const double2* A,
                             int64_t sam, int64_t sak, int conjA, const double2* B, int64_t sbk, int64_t sbn,
                             int conjB, double2* C, int64_t csm, int64_t csn, int beta, int64_t lower,
                             unsigned char* scratch, bool reuse_b, bool a_df) {
  constexpr size_t smem = 2 * (size_t)S * (OG_BM + OG_BNR) * OG_LD * 2;
  static DeviceFlags attr;  // per device, per slice count
  if (first_use_on_device(attr))
    cudaFuncSetAttribute(k_zgemm_sl<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const int64_t Mpad = (M + OG_BM - 1) / OG_BM * OG_BM, Npad = (Nb + 31) / 32 * 32;
  const int Kq = (int)((2 * K + 31) / 32 * 32);
  // B's slices first, so that a caller reusing them (reuse_b) keeps them in place
  __nv_bfloat16* Bs = (__nv_bfloat16*)scratch;
  int* cx = (int*)(scratch + al((size_t)2 * S * 2 * Npad * Kq));
  unsigned long long* cm = (unsigned long long*)((unsigned char*)cx + al(4 * (size_t)Npad));
  __nv_bfloat16* As = (__nv_bfloat16*)((unsigned char*)cm + al(8 * (size_t)Npad));
  int* rx = (int*)((unsigned char*)As + al((size_t)2 * S * Mpad * Kq));
  if (!reuse_b) {
    if (K <= 4 * OZ_KCHUNK) {
      (k_oz_slice_b<S><<<(unsigned)(Npad / 32), 256, 0, st>>>(B, sbk, sbn, conjB, (int)K, Nb, Kq, Npad, Bs, cx,
                                                             nullptr, (int)K), ++g_launches);
    } else {  // many rows: the column maxima first, then the slices of each chunk in parallel
      const unsigned kb = (unsigned)((K + OZ_KCHUNK - 1) / OZ_KCHUNK);
      cudaMemsetAsync(cm, 0, 8 * (size_t)Npad, st);
      (k_oz_colmax<<<dim3((unsigned)((Nb + 31) / 32), kb), 256, 0, st>>>(B, sbk, sbn, (int)K, Nb, OZ_KCHUNK, cm),
       ++g_launches);
      (k_oz_slice_b<S><<<dim3((unsigned)(Npad / 32), kb), 256, 0, st>>>(B, sbk, sbn, conjB, (int)K, Nb, Kq, Npad, Bs,
                                                                        cx, cm, OZ_KCHUNK), ++g_launches);
    }
  }
  if (a_df)
    (k_oz_slice_a<S, true><<<(unsigned)(Mpad / 8), 256, 0, st>>>(A, sam, sak, conjA, M, (int)K, Kq, Mpad, As, rx),
     ++g_launches);
  else
    (k_oz_slice_a<S, false><<<(unsigned)(Mpad / 8), 256, 0, st>>>(A, sam, sak, conjA, M, (int)K, Kq, Mpad, As, rx),
     ++g_launches);
  OzGemm q{As, Mpad, rx, Bs, Npad, cx, Kq, M, N, C, csm, csn, beta, lower};
  dim3 grid((unsigned)(Mpad / OG_BM), (unsigned)((N + 31) / 32));
  (k_zgemm_sl<S><<<grid, 256, smem, st>>>(q), ++g_launches);
}

bool zgemm_sliced(cudaStream_t st, int64_t M, int64_t N, int64_t K, const double2* A, int64_t sam, int64_t sak,
                  int conjA, const double2* B, int64_t sbk, int64_t sbn, int conjB, double2* C, int64_t csm,
                  int64_t csn, int beta, int64_t lower, unsigned char* scratch, size_t scratch_bytes, int64_t Nslice,
                  bool reuse_b, int slices, bool a_df) {
  if (M <= 0 || N <= 0) return true;
  const int64_t Nb = Nslice > N ? Nslice : N;  // columns of B that are sliced
  if (K <= 0 || (slices != 4 && slices != 5) || zgemm_sliced_bytes(M, Nb, K, slices) > scratch_bytes) return false;
  if (slices == 4)
    zgemm_sliced_run<4>(st, M, N, Nb, K, A, sam, sak, conjA, B, sbk, sbn, conjB, C, csm, csn, beta, lower, scratch,
                        reuse_b, a_df);
  else
    zgemm_sliced_run<5>(st, M, N, Nb, K, A, sam, sak, conjA, B, sbk, sbn, conjB, C, csm, csn, beta, lower, scratch,
                        reuse_b, a_df);
  return true;
}

void launch_slice_rows(cudaStream_t st, const double2* A, int64_t sam, int64_t sak, int64_t M, int K, int Kq,
                       int64_t Mpad, __nv_bfloat16* out, int* rexp) {
  (k_oz_slice_a<OZ_S, false><<<(unsigned)(Mpad / 8), 256, 0, st>>>(A, sam, sak, 0, M, K, Kq, Mpad, out, rexp),
   ++g_launches);
}

void launch_slice_cols(cudaStream_t st, const double2* B, int64_t sbk, int64_t sbn, int K, int64_t N, int Kq,
                       int64_t Npad, __nv_bfloat16* out, int* cexp) {
  (k_oz_slice_b<OZ_S><<<(unsigned)(Npad / 32), 256, 0, st>>>(B, sbk, sbn, 0, K, N, Kq, Npad, out, cexp, nullptr, K),
   ++g_launches);
}

// Fixed-order block sum of NV float-float values per thread (warp trees,
// then warps in order); thread t < nv of the block returns value t.
template <int NV>
__device__ __forceinline__ dfl block_df_sums(const dfl (&v)[NV], int nv, float2 (*sred)[NV]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    const dfl x = warp_df_sum(v[t]);
    if (lane == 0) sred[warp][t] = make_float2(x.hi, x.lo);
  }
  __syncthreads();
  dfl tot{0.f, 0.f};
  if ((int)threadIdx.x < nv) {
    tot = dfl{sred[0][threadIdx.x].x, sred[0][threadIdx.x].y};
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) tot = df_add(tot, dfl{sred[w][threadIdx.x].x, sred[w][threadIdx.x].y});
  }
  return tot;
}

// Per-row occupation sums of eta stored as float-float pairs (the sliced
// adjoint's adj.Hm): Hocc[r][t] = sum_A eta[r][A] [t occupied in A].  One
// block per row, threads over its strings; per thread NA cascaded sums
// (unrolled, predicated on the occupation bit), then a fixed-order block sum.
template <int NA>
__global__ void __launch_bounds__(256) k_hocc_df(const float2* __restrict__ H, DevList Ls, int na,
                                                 double* __restrict__ Hocc) {
  __shared__ float2 sred[8][NA];
  const int64_t r = blockIdx.x;
  const float2* h = H + r * Ls.n;
  OzSums acc[NA];
#pragma unroll
  for (int t = 0; t < NA; ++t) acc[t] = OzSums{0.f, 0.f};
  for (int64_t g = threadIdx.x; g < Ls.n; g += blockDim.x) {
    const float2 v = h[g];
    const uint64_t A = Ls.str[g];
#pragma unroll
    for (int t = 0; t < NA; ++t)
      if ((A >> t) & 1) acc[t].add(dfl{v.x, v.y});
  }
  dfl vals[NA];
#pragma unroll
  for (int t = 0; t < NA; ++t) vals[t] = acc[t].value();
  const dfl tot = block_df_sums<NA>(vals, na, sred);
  if ((int)threadIdx.x < na) Hocc[r * na + threadIdx.x] = df_to_double(tot);
}

void launch_hocc_df(cudaStream_t st, const float2* H, const DevList& L, int na, int64_t rows, double* Hocc) {
  if (rows <= 0) return;
  if (na <= 16) (k_hocc_df<16><<<(unsigned)rows, 256, 0, st>>>(H, L, na, Hocc), ++g_launches);
  else if (na <= 24) (k_hocc_df<24><<<(unsigned)rows, 256, 0, st>>>(H, L, na, Hocc), ++g_launches);
  else if (na <= 32) (k_hocc_df<32><<<(unsigned)rows, 256, 0, st>>>(H, L, na, Hocc), ++g_launches);
  else (k_hocc_df<64><<<(unsigned)rows, 256, 0, st>>>(H, L, na, Hocc), ++g_launches);
}

// |c_A|^2 / <c|c> as float-float pairs (the weights of class (2,2))
__global__ void k_c2df(const double2* __restrict__ c, int64_t n, const double2* __restrict__ g1,
                       float2* __restrict__ out) {
  const int64_t A = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (A >= n) return;
  const double2 v = c[A];
  const dfl d = df_from_double((v.x * v.x + v.y * v.y) / g1[0].x);
  out[A] = make_float2(d.hi, d.lo);
}

// Class (2,2), per row (i<j, a<b) over all strings A, in float-float (the
// FP64 kernel k_class22_rows computes the same sums): with w = |<ab||ij>|^2
// and f = w c2_A g(D), c2_A = |c_A|^2 / n,
//   hsum[row] = s sum_A df/dD,  P22[row] = s sum_A g c2_A (df/dw),
//   Hocc[row][t] = s sum_A df/dD [t in A],
// D = E0' - e_A - chi_ij^ab - U[a,A] - U[b,A] + U[i,A] + U[j,A].
template <int NA>
__global__ void __launch_bounds__(256)
k_class22_rows_df(DevList Ls, DevSpace sp, const float2* __restrict__ eAdf, const float2* __restrict__ Udf,
                  const float2* __restrict__ c2df, const double* __restrict__ g2, const double* __restrict__ epsh,
                  const double* __restrict__ G, const double* __restrict__ E0p, double b, double s,
                  double* __restrict__ hsum, double* __restrict__ Hocc, double* __restrict__ P22) {
  __shared__ float2 sred[8][NA + 2];
  __shared__ float2 sRow[2];  // E0' - chi, w
  const int64_t nvp = pairs(sp.nvc);
  const int64_t row = blockIdx.x;
  int iu, ju, au, bu;
  pair_decode(row / nvp, iu, ju);
  pair_decode(row % nvp, au, bu);
  if (threadIdx.x == 0) {
    const int gi = sp.cc[iu], gj = sp.cc[ju], ga = sp.vc[au], gb = sp.vc[bu];
    const double chi = -epsh[gi] - epsh[gj] + G[(int64_t)gi * sp.n + gj] + epsh[ga] + epsh[gb] +
                       G[(int64_t)ga * sp.n + gb] - G[(int64_t)gi * sp.n + ga] - G[(int64_t)gi * sp.n + gb] -
                       G[(int64_t)gj * sp.n + ga] - G[(int64_t)gj * sp.n + gb];
    const dfl base = df_from_double(*E0p - chi), w = df_from_double(g2[row]);
    sRow[0] = make_float2(base.hi, base.lo);
    sRow[1] = make_float2(w.hi, w.lo);
  }
  __syncthreads();
  const dfl base{sRow[0].x, sRow[0].y}, w{sRow[1].x, sRow[1].y};
  const bool shifted = b != 0.0;
  const dfl bb = df_from_double(b * b), b3 = df_from_double(3.0 * b * b);
  const float2* Ua = Udf + (int64_t)(sp.ncc + au) * Ls.n;
  const float2* Ub = Udf + (int64_t)(sp.ncc + bu) * Ls.n;
  const float2* Ui = Udf + (int64_t)iu * Ls.n;
  const float2* Uj = Udf + (int64_t)ju * Ls.n;
  OzSums ho[NA], hs{0.f, 0.f}, p22{0.f, 0.f};
#pragma unroll
  for (int t = 0; t < NA; ++t) ho[t] = OzSums{0.f, 0.f};
  for (int64_t A = threadIdx.x; A < Ls.n; A += blockDim.x) {
    const float2 e = eAdf[A], ua = Ua[A], ub = Ub[A], ui = Ui[A], uj = Uj[A], cc = c2df[A];
    dfl D = df_sub(base, dfl{e.x, e.y});
    D = df_sub(D, dfl{ua.x, ua.y});
    D = df_sub(D, dfl{ub.x, ub.y});
    D = df_add(D, dfl{ui.x, ui.y});
    D = df_add(D, dfl{uj.x, uj.y});
    const dfl c2{cc.x, cc.y};
    dfl gk, hw;  // g and w dg/dD
    if (!shifted) {
      gk = df_rcp(D);
      hw = df_mul(df_mul(w, gk), gk);
      hw = dfl{-hw.hi, -hw.lo};
    } else {
      const dfl D2 = df_sqr(D), D4 = df_sqr(D2);
      const dfl rq = df_rcp(df_add(D4, bb));
      gk = df_mul(df_mul(D, D2), rq);
      hw = df_mul(df_mul(df_mul(w, D2), df_sub(b3, D4)), df_sqr(rq));
    }
    const dfl hk = df_mul(c2, hw);
    hs.add(hk);
    p22.add(df_mul(gk, c2));
    const uint64_t bits = Ls.str[A];
#pragma unroll
    for (int t = 0; t < NA; ++t)
      if ((bits >> t) & 1) ho[t].add(hk);
  }
  dfl vals[NA + 2];
#pragma unroll
  for (int t = 0; t < NA; ++t) vals[t] = ho[t].value();
  vals[NA] = hs.value();
  vals[NA + 1] = p22.value();
  const int na = sp.n_act;
  // the block's sums: thread t < na gets Hocc[t]; NA and NA + 1 get hsum, P22
  const int t = threadIdx.x;
  const dfl tot = block_df_sums<NA + 2>(vals, NA + 2, sred);
  const dfl sd = df_from_double(s);
  if (t < na) Hocc[row * na + t] = df_to_double(df_mul(tot, sd));
  if (t == NA) hsum[row] = df_to_double(df_mul(tot, sd));
  if (t == NA + 1) P22[row] = df_to_double(df_mul(tot, sd));
}

void launch_class22_rows_df(cudaStream_t st, const DevList& L, const DevSpace& sp, const float2* eAdf,
                            const float2* Udf, const float2* c2df, const double* g2, const double* epsh,
                            const double* G, const double* E0p, double b, double s, int64_t rows, double* hsum,
                            double* Hocc, double* P22) {
  if (rows <= 0) return;
  const int na = sp.n_act;
#define E2_R22(NA_)                                                                                             \
  (k_class22_rows_df<NA_><<<(unsigned)rows, 256, 0, st>>>(L, sp, eAdf, Udf, c2df, g2, epsh, G, E0p, b, s, hsum, \
                                                          Hocc, P22),                                           \
   ++g_launches)
  if (na <= 16) E2_R22(16);
  else if (na <= 24) E2_R22(24);
  else if (na <= 32) E2_R22(32);
  else E2_R22(64);
#undef E2_R22
}

// Class (2,2) in float-float (the FP64 kernel k_class22's sum, same tiling
// and partial layout): per thread one string A, per block a pair of 8-wide
// virtual blocks and a core pair (i<j);
//   sum_{a<b in the blocks} |<ab||ij>|^2 |c_A|^2 g(D),
//   D = E0' - chi_ij - e_A + U[i,A] + U[j,A] - (alpha_a + U[a,A]) - (alpha_b + U[b,A]) - G_ab,
// the per-row quantities formed once per block in FP64 and kept as
// float-float pairs, the per-coupling work on the FP32 pipe.
__global__ void __launch_bounds__(256)
k_class22_df(DevList Ls, DevSpace sp, const float2* __restrict__ eAdf, const float2* __restrict__ Udf,
             const double2* __restrict__ c, const double* __restrict__ g2, const double* __restrict__ epsh,
             const double* __restrict__ G, const double* __restrict__ E0p, double b, int nvb,
             double* __restrict__ partial, unsigned long long* dmin, int64_t u0) {
  __shared__ float2 sGab[8][8], sG2[8][8], sAl[2][8], sBase;
  __shared__ float2 sW[8];
  // grid y: units u0 + blockIdx.y of (core pair z, virtual block pair y), u = z nyb + y
  const int64_t nyb = (int64_t)nvb * (nvb + 1) / 2;
  const int64_t u = u0 + blockIdx.y;
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
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < 64) {
    const int x = tid >> 3, y = tid & 7;
    const int a = ba * 8 + x, bq = bb * 8 + y;
    const bool ok = a < sp.nvc && bq < sp.nvc && a < bq;
    const dfl gab = df_from_double(ok ? G[(int64_t)sp.vc[a] * sp.n + sp.vc[bq]] : 0.0);
    const dfl w = df_from_double(ok ? g2[(int64_t)zp * nvp + pair_index(a, bq)] : 0.0);
    sGab[x][y] = make_float2(gab.hi, gab.lo);
    sG2[x][y] = make_float2(w.hi, w.lo);
  } else if (tid < 80) {
    const int k = tid - 64, side = k >> 3, x = k & 7;
    const int a = (side ? bb : ba) * 8 + x;
    double al = 0.0;
    if (a < sp.nvc) {
      const int ga = sp.vc[a];
      al = epsh[ga] - G[(int64_t)gi * sp.n + ga] - G[(int64_t)gj * sp.n + ga];
    }
    const dfl d = df_from_double(al);
    sAl[side][x] = make_float2(d.hi, d.lo);
  } else if (tid == 80) {
    const dfl d = df_from_double(*E0p + epsh[gi] + epsh[gj] - G[(int64_t)gi * sp.n + gj]);  // E0' - chi_ij
    sBase = make_float2(d.hi, d.lo);
  }
  __syncthreads();
  const int64_t A = blockIdx.x * (int64_t)blockDim.x + tid;
  dfl acc{0.f, 0.f};
  unsigned dmk = 0xFFFFFFFFu;
  if (A < Ls.n) {
    const bool shifted = b != 0.0;
    const dfl bbq = df_from_double(b * b);
    const float2 e = eAdf[A], ui = Udf[(int64_t)iu * Ls.n + A], uj = Udf[(int64_t)ju * Ls.n + A];
    dfl ct = df_sub(dfl{sBase.x, sBase.y}, dfl{e.x, e.y});
    ct = df_add(ct, dfl{ui.x, ui.y});
    ct = df_add(ct, dfl{uj.x, uj.y});
    dfl pb[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int bq = bb * 8 + k;
      pb[k] = dfl{0.f, 0.f};
      if (bq < sp.nvc) {
        const float2 u = Udf[(int64_t)(sp.ncc + bq) * Ls.n + A];
        pb[k] = df_add(dfl{sAl[1][k].x, sAl[1][k].y}, dfl{u.x, u.y});
      }
    }
    OzSums inner{0.f, 0.f};
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      const int a = ba * 8 + x;
      if (a >= sp.nvc) continue;
      const float2 u = Udf[(int64_t)(sp.ncc + a) * Ls.n + A];
      const dfl cx = df_sub(ct, df_add(dfl{sAl[0][x].x, sAl[0][x].y}, dfl{u.x, u.y}));
#pragma unroll
      for (int y = 0; y < 8; ++y) {
        const float2 w = sG2[x][y];
        if (w.x == 0.0f) continue;
        const dfl D = df_sub(df_sub(cx, pb[y]), dfl{sGab[x][y].x, sGab[x][y].y});
        dmk = min(dmk, fkey(D.hi));
        dfl g;
        if (!shifted) {
          g = df_rcp(D);
        } else {
          const dfl D2 = df_sqr(D);
          g = df_mul(df_mul(D, D2), df_rcp(df_add(df_sqr(D2), bbq)));
        }
        inner.add(df_mul(dfl{w.x, w.y}, g));
      }
    }
    const double2 cv = c[A];
    acc = df_mul(df_from_double(cv.x * cv.x + cv.y * cv.y), inner.value());
  }
  dmin_flush_f(dmin, dmk);
  acc = warp_df_sum(acc);
  if (lane == 0) sW[warp] = make_float2(acc.hi, acc.lo);
  __syncthreads();
  if (tid == 0) {
    dfl tot{sW[0].x, sW[0].y};
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) tot = df_add(tot, dfl{sW[w].x, sW[w].y});
    partial[u * gridDim.x + blockIdx.x] = df_to_double(tot);
  }
}

void launch_class22_df(cudaStream_t st, const DevList& L, const DevSpace& sp, const float2* eAdf, const float2* Udf,
                       const double2* c, const double* g2, const double* epsh, const double* G, const double* E0p,
                       double b, int nvb, int64_t ncp, double* partial, unsigned long long* dmin, int64_t u0,
                       int64_t u1) {
  // units u = z nyb + y over (core pair z, virtual block pair y), [u0, u1); y
  // of the grid holds at most 65535 of them per launch
  if (u1 < 0) u1 = ncp * ((int64_t)nvb * (nvb + 1) / 2);
  for (int64_t a = u0; a < u1; a += 65535) {
    dim3 grid((unsigned)((L.n + 255) / 256), (unsigned)std::min<int64_t>(65535, u1 - a));
    (k_class22_df<<<grid, 256, 0, st>>>(L, sp, eAdf, Udf, c, g2, epsh, G, E0p, b, nvb, partial, dmin, a),
     ++g_launches);
  }
}

}  // namespace e2
