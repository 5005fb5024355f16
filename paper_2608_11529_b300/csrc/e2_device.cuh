// Device helpers shared by the forward and adjoint kernels.
#pragma once
#include <cuda_runtime.h>

#include "e2_common.cuh"

namespace e2 {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// |x| as an ordered integer key: the bit pattern without its sign (for
// non-negative doubles the integer order is the numeric order; NaN keys sit
// above +inf, so they never lower a minimum).
__device__ __forceinline__ unsigned long long dkey(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFULL;
}
// The same for a float (the high part of a float-float denominator).
__device__ __forceinline__ unsigned fkey(float x) { return __float_as_uint(x) & 0x7FFFFFFFu; }

// Smallest |D| key of the warp into *slot with one atomicMin per warp
// (slot null: nothing).  Every lane of the warp must call it.
__device__ __forceinline__ void dmin_flush(unsigned long long* slot, unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (slot && (threadIdx.x & 31) == 0 && v != ~0ULL) atomicMin(slot, v);
}
// A float key (fkey) converted to the double key of the same magnitude.
__device__ __forceinline__ void dmin_flush_f(unsigned long long* slot, unsigned v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (slot && (threadIdx.x & 31) == 0 && v != 0xFFFFFFFFu) atomicMin(slot, dkey((double)__uint_as_float(v)));
}

__device__ __forceinline__ int popc_below(uint64_t A, int t) {
  return __popcll(t ? (A & ((1ull << t) - 1)) : 0ull);
}

// 1/d: single-precision seed refined by two Newton-Raphson steps
// (x <- x (2 - d x)); each step squares the relative error, 2^-23 -> 2^-46
// -> below double rounding.  Valid for 1e-30 < |d| < 1e30.
__device__ __forceinline__ double rcp_nr(double d) {
  double r = (double)__frcp_rn(__double2float_rn(d));
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}

// Weight g(D) of the Epstein-Nesbet term f = v g(D): g = 1/D, or with the
// imaginary level shift the real part of 1/(D + i b/D) = D^3/(D^4 + b^2)
// (Sec. 2.6).  g is also df/dv.
__device__ __forceinline__ double en_g(double D, double b) {
  if (b == 0.0) return rcp_nr(D);
  const double D2 = D * D;
  return D * D2 * rcp_nr(fma(D2, D2, b * b));
}

// Reciprocals of four values with one reciprocal (simultaneous inversion:
// prefix products, one rcp_nr, back-substitution; 15 FP64 operations for
// four instead of 24).  When the product's magnitude leaves [2^-99, 2^99)
// (rcp_nr seeds in single precision; a NaN or an infinity also leaves it)
// the four are inverted one by one.  The range test reads the exponent
// field with integer operations, off the FP64 pipe.
__device__ __forceinline__ void rcp4(const double (&q)[4], double (&r)[4]) {
  const double p1 = q[0] * q[1], p2 = p1 * q[2], p3 = p2 * q[3];
  const unsigned ex = ((unsigned)__double2hiint(p3) >> 20) & 0x7FFu;  // biased exponent
  if (ex - 924u < 1122u - 924u) {
    double s = rcp_nr(p3);
    r[3] = s * p2;
    s *= q[3];
    r[2] = s * p1;
    s *= q[2];
    r[1] = s * q[0];
    r[0] = s * q[1];
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) r[k] = rcp_nr(q[k]);
  }
}

// The quantity whose reciprocal g(D) needs: D, or D^4 + b^2 with the level shift.
__device__ __forceinline__ double en_q(double D, double b) {
  if (b == 0.0) return D;
  const double D2 = D * D;
  return fma(D2, D2, b * b);
}

// g(D) from r = 1 / en_q(D, b); the same arithmetic in every pass that uses it.
__device__ __forceinline__ double en_g_r(double D, double b, double r) {
  if (b == 0.0) return r;
  return D * (D * D) * r;
}

// df/dv and df/dD of f(v, D) = v g(D) from r = 1 / en_q(D, b); g is en_g_r.
__device__ __forceinline__ void en_derivs_r(double v, double D, double b, double r, double& g, double& h) {
  if (b == 0.0) {
    g = r;
    h = -v * r * r;
    return;
  }
  const double D2 = D * D;
  g = D * D2 * r;
  h = v * D2 * fma(3.0 * b, b, -D2 * D2) * r * r;
}

// df/dv and df/dD of f(v, D) = v g(D); g bitwise equal to en_g.
__device__ __forceinline__ void en_derivs(double v, double D, double b, double& g, double& h) {
  if (b == 0.0) {
    const double r = rcp_nr(D);
    g = r;
    h = -v * r * r;
    return;
  }
  const double D2 = D * D, r = rcp_nr(fma(D2, D2, b * b));
  g = D * D2 * r;
  h = v * D2 * fma(3.0 * b, b, -D2 * D2) * r * r;
}

__device__ __forceinline__ void pair_decode(int64_t e, int& x, int& y) {
  int64_t yy = (int64_t)((1.0 + sqrt(1.0 + 8.0 * (double)e)) * 0.5);
  while (yy > 1 && yy * (yy - 1) / 2 > e) --yy;
  while ((yy + 1) * yy / 2 <= e) ++yy;
  y = (int)yy;
  x = (int)(e - yy * (yy - 1) / 2);
}

__device__ __forceinline__ int pair_index(int x, int y) { return y * (y - 1) / 2 + x; }  // x < y


// Global spinor indices (p, q, r, s) of entry (row, col) of an integral block
// <pq||rs> (see IntMode); returns true for the one-body column of INT_W11
// (f_pq, with q in place of the occupied index).
__device__ inline bool int_indices(int mode, const DevSpace& sp, int64_t row, int col, int& p, int& q, int& r, int& s) {
  const int na = sp.n_act, a0 = sp.a0, nvp = (int)pairs(sp.nvc), ntp = (int)pairs(na);
  int x, y;
  p = q = r = s = 0;
  switch (mode) {
    case INT_W02:
      pair_decode(row, x, y);
      p = sp.vc[x]; q = sp.vc[y];
      pair_decode(col, x, y);
      r = a0 + x; s = a0 + y;
      break;
    case INT_W12: {
      const int i = (int)(row / nvp);
      pair_decode(row % nvp, x, y);
      p = sp.vc[x]; q = sp.vc[y]; r = sp.cc[i]; s = a0 + col;
    } break;
    case INT_W21: {
      const int a = (int)(row % sp.nvc);
      pair_decode(row / sp.nvc, x, y);
      p = sp.vc[a]; q = a0 + col; r = sp.cc[x]; s = sp.cc[y];
    } break;
    case INT_W11: {
      const int i = (int)(row / sp.nvc), a = (int)(row % sp.nvc);
      if (col == 0) {
        p = sp.vc[a]; q = sp.cc[i];
        return true;
      }
      const int t = (col - 1) / na, u = (col - 1) % na;
      p = sp.vc[a]; q = a0 + t; r = sp.cc[i]; s = a0 + u;
    } break;
    case INT_W20:
      pair_decode(row, x, y);
      r = sp.cc[x]; s = sp.cc[y];
      pair_decode(col, x, y);
      p = a0 + x; q = a0 + y;
      break;
    case INT_G22:
    case INT_G22C:
      pair_decode(row, x, y);
      r = sp.cc[x]; s = sp.cc[y];
      pair_decode(col, x, y);
      p = sp.vc[x]; q = sp.vc[y];
      break;
    case INT_X01: {
      const int u = col / ntp;
      pair_decode(col % ntp, x, y);
      p = sp.vc[row]; q = a0 + u; r = a0 + x; s = a0 + y;
    } break;
    case INT_X10: {
      const int vv = col % na;
      pair_decode(col / na, x, y);
      p = a0 + x; q = a0 + y; r = sp.cc[row]; s = a0 + vv;
    } break;
    case INT_X00:
      pair_decode(row, x, y);
      p = a0 + x; q = a0 + y;
      pair_decode(col, x, y);
      r = a0 + x; s = a0 + y;
      break;
  }
  return false;
}

// Colex rank of a substring with k set bits: sum_j C(t_j, j), j = 1..k.
__device__ __forceinline__ int64_t colex_rank(uint64_t bits, const int64_t* __restrict__ binom) {
  int64_t r = 0;
  int j = 0;
  while (bits) {
    int t = __ffsll((long long)bits) - 1;
    bits &= bits - 1;
    ++j;
    r += binom[t * kBinomN + j];
  }
  return r;
}

__device__ __forceinline__ uint64_t colex_unrank(int64_t rank, int k, int size, const int64_t* __restrict__ binom) {
  uint64_t out = 0;
  int t = size - 1;
  for (int j = k; j >= 1; --j) {
    while (binom[t * kBinomN + j] > rank) --t;
    out |= 1ull << t;
    rank -= binom[t * kBinomN + j];
    --t;
  }
  return out;
}

// Position of string A in list Ls, or -1 when A's pattern is not in the list.
__device__ __forceinline__ int64_t list_addr(const DevList& Ls, const DevDas& das, const int64_t* __restrict__ binom,
                                             uint64_t A) {
  if (Ls.key2off == nullptr) return -1;
  int key = 0;
  int occ[E2_MAX_DAS];
  for (int s = 0; s < das.n_das; ++s) {
    uint64_t m = ((das.size[s] == 64) ? ~0ull : ((1ull << das.size[s]) - 1)) << das.off[s];
    occ[s] = __popcll(A & m);
    key += occ[s] * das.keymul[s];
  }
  int64_t off = Ls.key2off[key];
  if (off < 0) return -1;
  int64_t stride = 1;
  for (int s = 0; s < das.n_das; ++s) {
    uint64_t sub = (A >> das.off[s]) & ((das.size[s] == 64) ? ~0ull : ((1ull << das.size[s]) - 1));
    off += colex_rank(sub, binom) * stride;
    stride *= binom[das.size[s] * kBinomN + occ[s]];
  }
  return off;
}

// Fixed-order block sum of a per-thread double; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < nw; ++k) t += sh[k];
  return t;
}

// One m16n8k8 FP64 tensor-pipe product: c += a b (a: 16x8 row fragment,
// b: 8x8 column fragment, c: 16x8 accumulator fragment).
__device__ __forceinline__ void mma_f64(double (&c)[4], const double (&a)[4], const double (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(b[0]), "d"(b[1]));
}

// D (16x8) += A (16x4, row) * B (4x8, col) in FP64: a[0] = A[g][tq],
// a[1] = A[g+8][tq], b = B[tq][g] (g = lane / 4, tq = lane % 4); C as for k = 8.
__device__ __forceinline__ void mma_f64_k4(double (&c)[4], const double (&a)[2], double b) {
  asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
               : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
               : "d"(a[0]), "d"(a[1]), "d"(b));
}

// <A| H - E_O |Psi> for an n_elec-electron string A with no core hole or
// virtual particle: sum_{tu} f_tu D^{t+u}_A + sum_{t<u in A} s(A;t,u)
// sum_{v<w} <tu||vw> D^{vw}_{A-t-u}.  Class (0,0) evaluates it on strings of
// non-reference patterns; the reference solver evaluates it on P (sigma = H c).
__device__ inline double2 active_sigma(uint64_t A, const DevList& L11, const DevList& L02, const DevDas& das,
                                const DevSpace& sp, const int64_t* __restrict__ binom, const double2* __restrict__ DTDU,
                                const double2* __restrict__ DTU, const double2* __restrict__ X00,
                                const double2* __restrict__ f) {
  const int na = sp.n_act, ntp = (int)pairs(na);
  double2 V = make_double2(0.0, 0.0);
  int64_t a11 = list_addr(L11, das, binom, A);
  if (a11 >= 0)
    for (int t = 0; t < na; ++t)
      for (int u = 0; u < na; ++u)
        V = cfma(f[(int64_t)(sp.a0 + t) * sp.n_occ + sp.a0 + u], DTDU[(int64_t)(1 + t * na + u) * L11.n + a11], V);
  for (uint64_t xu = A; xu; xu &= xu - 1) {
    const int u = __ffsll((long long)xu) - 1;
    for (uint64_t xt = A & ((1ull << u) - 1); xt; xt &= xt - 1) {
      const int t = __ffsll((long long)xt) - 1;
      const uint64_t B = A & ~(1ull << t) & ~(1ull << u);
      const int64_t a02 = list_addr(L02, das, binom, B);
      if (a02 < 0) continue;
      const double2* Xr = X00 + (int64_t)pair_index(t, u) * ntp;
      double2 s = make_double2(0.0, 0.0);
      for (int w = 1; w < na; ++w) {
        if ((B >> w) & 1) continue;
        for (int v = 0; v < w; ++v) {
          if ((B >> v) & 1) continue;
          const int vw = pair_index(v, w);
          s = cfma(Xr[vw], DTU[(int64_t)vw * L02.n + a02], s);
        }
      }
      if ((popc_below(B, u) + popc_below(B, t)) & 1) s = make_double2(-s.x, -s.y);
      V.x += s.x;
      V.y += s.y;
    }
  }
  return V;
}

}  // namespace e2
