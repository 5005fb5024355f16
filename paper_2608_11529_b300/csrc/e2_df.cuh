// Double-word single precision ("float-float"): a value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant bits.
// On this part the FP32 pipe issues about 70 times as many operations per
// clock as the FP64 pipe, so a float-float operation of 3 to 20 FP32
// instructions costs a fraction of one FP64 instruction.
//
// The building blocks are the classical error-free transformations:
//   two_sum       Knuth's TwoSum: s + e = a + b exactly (6 operations);
//   fast_two_sum  Dekker's FastTwoSum, valid when |a| >= |b| or a = 0;
//   two_prod      p + e = a * b exactly, with one fused multiply-add.
// The double-word sums and products follow the algorithms analysed by Joldes,
// Muller and Popescu ("Tight and rigorous error bounds for basic building
// blocks of double-word arithmetic", ACM TOMS 44, 2017): the accurate sum
// (relative error below 3u^2 + 13u^3, u = 2^-24), and a product with one
// fused multiply-add per cross term (relative error below 5u^2).
//
// Every rounding is explicit (__fadd_rn, __fmul_rn, __fmaf_rn), so the
// compiler neither contracts nor reorders these sequences.
#pragma once
#include <cuda_runtime.h>

namespace e2 {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfl{s, e};
}

__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfl{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return dfl{p, __fmaf_rn(a, b, -p)};
}

// a + b, both double-word (accurate sum)
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const dfl s = two_sum(a.hi, b.hi);
  const dfl t = two_sum(a.lo, b.lo);
  const dfl v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

// a - b
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, dfl{-b.hi, -b.lo}); }

// a + b with b a float
__device__ __forceinline__ dfl df_add_f(dfl a, float b) {
  const dfl s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(a.lo, s.lo));
}

// a * b, both double-word
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const dfl p = two_prod(a.hi, b.hi);
  float e = __fmul_rn(a.hi, b.lo);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p.hi, __fadd_rn(p.lo, e));
}

// a * b with b a float
__device__ __forceinline__ dfl df_mul_f(dfl a, float b) {
  const dfl p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// a^2
__device__ __forceinline__ dfl df_sqr(dfl a) {
  const dfl p = two_prod(a.hi, a.hi);
  return fast_two_sum(p.hi, __fmaf_rn(__fadd_rn(a.hi, a.hi), a.lo, p.lo));
}

// a * 2^k (exact while the result stays a normal float)
__device__ __forceinline__ dfl df_scale(dfl a, float two_k) { return dfl{__fmul_rn(a.hi, two_k), __fmul_rn(a.lo, two_k)}; }

// 1/a: a single-precision reciprocal r (relative error about 2^-23) and one
// Newton step carried in double-word arithmetic, 1/a = r + r (1 - a r): the
// residual 1 - a r is formed exactly from the product a.hi * r, so the step
// squares the seed's error to about 2^-46.
__device__ __forceinline__ dfl df_rcp(dfl a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a.hi));
  const dfl p = two_prod(a.hi, r);                         // a.hi r exactly
  float e = __fsub_rn(1.0f, p.hi);                          // exact: p.hi is within 2^-22 of 1
  e = __fsub_rn(e, p.lo);
  e = __fmaf_rn(-a.lo, r, e);                               // - a.lo r
  return fast_two_sum(r, __fmul_rn(r, e));
}

// Double precision in and out (per-string tables are converted once; a
// kernel that converts per coupling pays FP64 throughput).
__host__ __device__ __forceinline__ dfl df_from_double(double x) {
  const float h = (float)x;
  return dfl{h, (float)(x - (double)h)};
}
__host__ __device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

}  // namespace e2
