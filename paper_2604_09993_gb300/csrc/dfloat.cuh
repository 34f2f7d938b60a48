// dfloat.cuh — float-float ("double-single") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum h + l of two floats with |l| a few ulp(h)
// at most, about 47 significand bits.  On this GPU one FP64-pipe
// instruction takes the issue time of ~64 FP32 instructions, so the
// kernels evaluate the right-hand side of their RK stages (angle chain,
// slopes, penalty integrands) in this arithmetic and keep FP64 only for the
// accumulation of the state and of the penalty state across substeps.
//
// Algorithms (all published, written here from their definitions):
//  * TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly, any order;
//  * Fast2Sum (Dekker 1971): the same for |a| >= |b|;
//  * TwoProd with an FMA: p + e = a b exactly (e = fma(a, b, -p));
//  * the sum of two float-float numbers in the "sloppy" form (TwoSum of
//    the high parts, the low parts added in FP32, one Fast2Sum): its
//    absolute error is <= 4u^2 (|x| + |y|), u = 2^-24, which is what these
//    kernels need (errors on the scale of the operands), though under
//    cancellation it has no relative bound;
//  * the product with an FMA (TwoProd of the high parts plus the two cross
//    terms), left unnormalized: relative error <= 12u^2 for operands whose
//    low part is below one ulp of the high part, the result's low part a few
//    ulp of its high part at most; every sum renormalizes.
// (Joldes, Muller and Popescu, ACM TOMS 44(2), 2017, analyse these forms.)
// The device versions use the _rn intrinsics so that the compiler never
// contracts a product and a sum into one FMA, which would break the exact
// error terms; the host versions (tests) are compiled without contraction.
#pragma once

#if defined(__CUDACC__)
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#include <cmath>
#include <cstdint>
#include <cstring>
#endif

namespace ciscvx {

struct dflt {
  float h, l;
};

DF_HD float f_add(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
DF_HD float f_sub(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
DF_HD float f_mul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
DF_HD float f_fma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

DF_HD dflt df_make(float h) { return dflt{h, 0.0f}; }

// Knuth's TwoSum.
DF_HD dflt two_sum(float a, float b) {
  const float s = f_add(a, b);
  const float bb = f_sub(s, a);
  const float e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
  return dflt{s, e};
}
// Dekker's Fast2Sum (|a| >= |b| or a = 0).
DF_HD dflt fast_two_sum(float a, float b) {
  const float s = f_add(a, b);
  return dflt{s, f_sub(b, f_sub(s, a))};
}
// TwoProd with an FMA.
DF_HD dflt two_prod(float a, float b) {
  const float p = f_mul(a, b);
  return dflt{p, f_fma(a, b, -p)};
}

DF_HD dflt df_neg(dflt x) { return dflt{-x.h, -x.l}; }
// Exact scaling by a power of two (no overflow or underflow in this use).
DF_HD dflt df_scale(dflt x, float p2) { return dflt{f_mul(x.h, p2), f_mul(x.l, p2)}; }

// x + y (sloppy form, renormalized).
DF_HD dflt df_add(dflt x, dflt y) {
  const dflt s = two_sum(x.h, y.h);
  return fast_two_sum(s.h, f_add(s.l, f_add(x.l, y.l)));
}
DF_HD dflt df_sub(dflt x, dflt y) { return df_add(x, df_neg(y)); }
// x + f, f a float.
DF_HD dflt df_add_f(dflt x, float f) {
  const dflt s = two_sum(x.h, f);
  return fast_two_sum(s.h, f_add(s.l, x.l));
}
// x y (unnormalized).
DF_HD dflt df_mul(dflt x, dflt y) {
  dflt p = two_prod(x.h, y.h);
  p.l = f_fma(x.h, y.l, p.l);
  p.l = f_fma(x.l, y.h, p.l);
  return p;
}
// x f, f a float (unnormalized).
DF_HD dflt df_mul_f(dflt x, float f) {
  dflt p = two_prod(x.h, f);
  p.l = f_fma(x.l, f, p.l);
  return p;
}
// x^2 (unnormalized)
DF_HD dflt df_sqr(dflt x) {
  dflt p = two_prod(x.h, x.h);
  p.l = f_fma(f_add(x.h, x.h), x.l, p.l);
  return p;
}

// Constants 1/n as float-float, formed at compile time from the double value.
#define DF_CONST(v) (::ciscvx::dflt{(float)(v), (float)((v) - (double)(float)(v))})

// ---------------------------------------------------------------------------
// Conversions between FP64 and float-float.  On this part a conversion
// instruction takes an FP64-pipe slot, so the split works on the bit
// patterns (integer pipe): the high part keeps the sign, the rebiased
// exponent and the top 23 fraction bits (round toward zero); the low part is
// the remaining 29 fraction bits, normalized into a float (its last 5 bits
// truncated), so |l| < ulp(h).  |x - (h + l)| <= 2^-47 |x| for normal x
// with |x| in
// [2^-90, 2^127]; outside that range the low part is flushed to zero and the
// high part is the FP32 value toward zero (0 below 2^-126).
// ---------------------------------------------------------------------------
#if defined(__CUDACC__)
__device__ __forceinline__ unsigned dbl_hi(double x) { return (unsigned)__double2hiint(x); }
__device__ __forceinline__ unsigned dbl_lo(double x) { return (unsigned)__double2loint(x); }
__device__ __forceinline__ float bits_f(unsigned u) { return __uint_as_float(u); }
__device__ __forceinline__ int clz32(unsigned v) { return __clz((int)v); }
#define DF_DEV __device__ __forceinline__
#else
inline unsigned dbl_hi(double x) { uint64_t u; std::memcpy(&u, &x, 8); return (unsigned)(u >> 32); }
inline unsigned dbl_lo(double x) { uint64_t u; std::memcpy(&u, &x, 8); return (unsigned)u; }
inline float bits_f(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
inline int clz32(unsigned v) { return v ? __builtin_clz(v) : 32; }
#define DF_DEV inline
#endif

DF_DEV dflt df_split(double x) {
  const unsigned hi = dbl_hi(x), lo = dbl_lo(x);
  const unsigned sign = hi & 0x80000000u;
  const int E = (int)((hi >> 20) & 0x7ffu);  // biased FP64 exponent
  const int eh = E - 896;                     // FP32 biased exponent of the high part
  unsigned hb = sign | ((unsigned)eh << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  if (eh <= 0) hb = sign;
  if (eh >= 255) hb = sign | 0x7f800000u | ((((hi & 0xfffffu) | lo) != 0u && E == 0x7ff) ? 0x400000u : 0u);
  // low part: r * 2^(E - 1075), r = the low 29 fraction bits
  const unsigned r = lo & 0x1fffffffu;
  unsigned lb = 0u;
  if (r != 0u && eh > 0 && eh < 255) {
    const int p = 31 - clz32(r);      // leading bit of r, 0..28
    const int el = p + E - 948;       // FP32 biased exponent of the low part
    const unsigned m = (p >= 23) ? (r >> (p - 23)) : (r << (23 - p));
    if (el > 0) lb = sign | ((unsigned)el << 23) | (m & 0x7fffffu);
  }
  return dflt{bits_f(hb), bits_f(lb)};
}

// ---------------------------------------------------------------------------
// sin d and 1 - cos d of a small angle increment d, from their Taylor
// series with the leading terms in float-float and the tail in FP32.
//  * short tier, |d| <= 0.02: sin d = d - d q, q = x/6 - x^2/120 + x^3/5040,
//    1 - cos d = x/2 - x^2/24 + x^3/720, x = d^2 (truncation <= 3e-16);
//  * long tier, |d| <= 0.2: q through x^5 and 1 - cos d through x^5, with
//    x/6, x^2/120, x^2/24 and x^3/720 in float-float (truncation <= 2e-16).
// Absolute error of either result <= 5e-15 for d exact in float-float (the
// FP32 tail terms dominate).
// ---------------------------------------------------------------------------
DF_HD void sin_vers_short(dflt d, dflt& sn, dflt& vc) {
  const dflt x = df_sqr(d);
  const float xh = x.h;
  // q = x/6 - x^2 (1/120 - x/5040)
  const float tq = f_mul(f_mul(xh, xh), f_fma(xh, (float)(1.0 / 5040.0), (float)(-1.0 / 120.0)));
  const dflt q = df_add_f(df_mul(x, DF_CONST(1.0 / 6.0)), tq);
  sn = df_sub(d, df_mul(d, q));
  // 1 - cos d = x/2 - x^2 (1/24 - x/720)
  const float tv = f_mul(f_mul(xh, xh), f_fma(xh, (float)(1.0 / 720.0), (float)(-1.0 / 24.0)));
  vc = df_add_f(df_scale(x, 0.5f), tv);
}

DF_HD void sin_vers_long(dflt d, dflt& sn, dflt& vc) {
  const dflt x = df_sqr(d);
  const float xh = x.h;
  const float x2 = f_mul(xh, xh);
  // q = x (1/6 - x/120) + x^3 (1/5040 - x/362880 + x^2/39916800)
  const float tq = f_mul(f_mul(x2, xh),
                         f_fma(xh, f_fma(xh, (float)(1.0 / 39916800.0), (float)(-1.0 / 362880.0)),
                               (float)(1.0 / 5040.0)));
  const dflt q = df_add_f(df_mul(x, df_sub(DF_CONST(1.0 / 6.0), df_mul(x, DF_CONST(1.0 / 120.0)))), tq);
  sn = df_sub(d, df_mul(d, q));
  // 1 - cos d = x/2 - x^2 (1/24 - x/720) - x^4 (1/40320 - x/3628800)
  const float tv = f_mul(f_mul(x2, x2), f_fma(xh, (float)(1.0 / 3628800.0), (float)(-1.0 / 40320.0)));
  const dflt inner = df_sub(DF_CONST(1.0 / 24.0), df_mul(x, DF_CONST(1.0 / 720.0)));
  vc = df_add_f(df_sub(df_scale(x, 0.5f), df_mul(df_sqr(x), inner)), tv);
}

// Pseudo-Huber ramp h(z) = sqrt(1 + p^2) - 1, p = max(z, 0), in float-float:
// a = 1 + p^2, y0 = sqrt(a_h) (FP32, correctly rounded), and one correction
// (a - y0^2) / (2 y0) with the residual formed exactly by TwoProd; the
// result's error is <= 3e-14 max(1, h) for |z| <= 10 (the cancellation in
// sqrt(a) - 1 for small p only affects values far below that bound).
DF_HD dflt huber_df(dflt z) {
  if (!(z.h > 0.0f)) return dflt{0.0f, 0.0f};
  const dflt a = df_add_f(df_sqr(z), 1.0f);
#if defined(__CUDA_ARCH__)
  const float y0 = __fsqrt_rn(a.h);
  const float r = rsqrtf(a.h);
#else
  const float y0 = std::sqrt(a.h);
  const float r = 1.0f / std::sqrt(a.h);
#endif
  const dflt q = two_prod(y0, y0);
  const float e = f_add(f_sub(f_sub(a.h, q.h), q.l), a.l);
  const float y1 = f_mul(f_mul(e, 0.5f), r);
  const dflt t = two_sum(y0, -1.0f);
  return fast_two_sum(t.h, f_add(t.l, y1));
}

}  // namespace ciscvx
