// df64.cuh -- double-float ("df64") arithmetic on the FP32 pipe for FP64-accurate results.
//
// GB300 issues FP32 operations at 61 times its FP64 rate (measured 72.4 vs 1.19 TFLOP/s),
// so the FP64-mode event kernels carry their long polynomial and transcendental chains as
// unevaluated pairs hi + lo of floats (48-bit significands, relative rounding ~2^-46) and
// keep FP64 for range reductions, the inputs and the results.  Error-free transformations:
// Knuth's TwoSum, Dekker's FastTwoSum, and the FMA product error (exact for binary32).
// __fadd_rn / __fmul_rn / __fmaf_rn keep the compiler from contracting or reordering them.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace gfi {

struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 df_add(F2 a, F2 b) {
  const F2 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ F2 df_neg(F2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ F2 df_sub(F2 a, F2 b) { return df_add(a, df_neg(b)); }
// product as an unnormalised pair (p, e): p = fl(a.hi b.hi), e = its error + cross terms
__device__ __forceinline__ F2 df_mul_raw(F2 a, F2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return {p, e};
}
__device__ __forceinline__ F2 df_mul(F2 a, F2 b) {
  const F2 r = df_mul_raw(a, b);
  return fast_two_sum(r.hi, r.lo);
}
__device__ __forceinline__ F2 df_mul_f(F2 a, float b) {
  const float p = __fmul_rn(a.hi, b);
  return fast_two_sum(p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p)));
}
// a / b: float quotient, its remainder in df64, one correction
__device__ __forceinline__ F2 df_div(F2 a, F2 b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const F2 r = df_sub(a, df_mul_f(b, q1));
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return fast_two_sum(q1, q2);
}
__device__ __forceinline__ F2 df_from(double v) {
  const float hi = __double2float_rn(v);
  return {hi, __double2float_rn(v - (double)hi)};
}
__device__ __forceinline__ double df_to(F2 a) { return (double)a.hi + (double)a.lo; }

// Constant c as a df64 pair, formed at compile time.
struct DFC {
  float hi, lo;
  __host__ __device__ constexpr DFC(double c) : hi((float)c), lo((float)(c - (double)(float)c)) {}
  __device__ __forceinline__ operator F2() const { return {hi, lo}; }
};

// ---- natural logarithm -----------------------------------------------------------------
// x = m 2^e with m in [1/sqrt2, sqrt2) (exponent bits, integer pipe); log m = 2 atanh(s),
// s = (m - 1)/(m + 1), |s| <= 0.1716, by its odd series to s^21 in df64; e ln2 in FP64.
// Absolute error ~1e-15 for normal positive x; other x go to the library log.
__device__ __forceinline__ double df_log(double x) {
  if (!(x >= 2.2250738585072014e-308 && x < 1.7976931348623157e308)) return log(x);
  long long b = __double_as_longlong(x);
  int e = (int)((b >> 52) & 0x7ff) - 1023;
  b = (b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL;  // m in [1, 2)
  if (b > 0x3ff6a09e667f3bccLL) {                         // m > sqrt 2: halve it
    b -= 0x0010000000000000LL;
    e += 1;
  }
  const F2 m = df_from(__longlong_as_double(b));
  const F2 s = df_div(df_add(m, F2{-1.f, 0.f}), df_add(m, F2{1.f, 0.f}));
  const F2 s2 = df_mul(s, s);
  constexpr DFC c[11] = {1.0, 1.0 / 3, 1.0 / 5, 1.0 / 7, 1.0 / 9, 1.0 / 11,
                         1.0 / 13, 1.0 / 15, 1.0 / 17, 1.0 / 19, 1.0 / 21};
  F2 p = c[10];
#pragma unroll
  for (int k = 9; k >= 0; --k) p = df_add(df_mul(p, s2), c[k]);
  const double lm = df_to(df_mul(df_mul_f(s, 2.f), p));
  return fma((double)e, 0.69314718055994530942, lm);
}

// ---- exponential ----------------------------------------------------------------------
// u = k ln2 + r (k = rint(u / ln2), r by one FP64 FMA, |r| <= 0.347); e^r by its Taylor
// series to r^14/14! in df64; 2^k by the exponent bits.  Relative error ~1e-15 for
// -700 < u < 700; other u go to the library exp.
__device__ __forceinline__ double df_exp(double u) {
  if (!(u > -700.0 && u < 700.0)) return exp(u);
  const double k = rint(u * 1.4426950408889634074);
  const F2 r = df_from(fma(-k, 0.69314718055994530942, u));
  constexpr DFC c[15] = {1.0,
                         1.0,
                         1.0 / 2,
                         1.0 / 6,
                         1.0 / 24,
                         1.0 / 120,
                         1.0 / 720,
                         1.0 / 5040,
                         1.0 / 40320,
                         1.0 / 362880,
                         1.0 / 3628800,
                         1.0 / 39916800,
                         1.0 / 479001600,
                         1.0 / 6227020800.0,
                         1.0 / 87178291200.0};
  F2 p = c[14];
#pragma unroll
  for (int j = 13; j >= 0; --j) p = df_add(df_mul(p, r), c[j]);
  const double v = df_to(p);
  return __longlong_as_double(__double_as_longlong(v) + ((long long)k << 52));
}

}  // namespace gfi
