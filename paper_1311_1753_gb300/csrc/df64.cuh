// df64.cuh -- double-float ("df64") arithmetic on the FP32 pipe for FP64-accurate results.
//
// GB300 issues FP32 operations at 64 times its FP64 rate (measured 72.4 vs 1.19 TFLOP/s),
// so the FP64-mode event kernels carry their arithmetic as unevaluated pairs hi + lo of
// floats (48-bit significands, relative rounding ~2^-47): data enter by an exact-to-2^-48
// bit split, range reductions of exp and log work on pairs with split constants, and
// FP64 is left for the exact differences of data and constants, the cold paths and the
// cross-thread sums.  Error-free transformations: Knuth's TwoSum, Dekker's FastTwoSum,
// and the FMA product error (exact for binary32).  __fadd_rn / __fmul_rn / __fmaf_rn keep
// the compiler from contracting or reordering them.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
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

// df_from out of line, for the rare inputs of the bit splits below: inline, the compiler
// may predicate its two conversions and FP64 subtraction into every call, and predicated-
// off FP64 instructions still occupy GB300's narrow FP64 pipe.
static __device__ __noinline__ F2 df_from_cold(double v) { return df_from(v); }

// d as a pair without FP64 conversions (integer pipe and a few FP32 operations): hi is d
// rounded to 24 significant bits (round half up on the magnitude), lo the remainder
// (at most 28 bits and a sign) rounded to 24, so hi + lo equals d to 2^-48 relative.
// |d| outside [2^-74, 2^126) (and 0) takes the conversion path.
__device__ __forceinline__ F2 df_split(double d) {
  const long long b = __double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e < 949 || e > 1149) return df_from_cold(d);
  const unsigned sign = (unsigned)((unsigned long long)b >> 32) & 0x80000000u;
  const unsigned up = (unsigned)(b >> 28) & 1u;  // top bit of the remainder: round up
  const float hi = __uint_as_float((sign | ((unsigned)(e - 896) << 23) |
                                    ((unsigned)(b >> 29) & 0x7fffffu)) + up);
  // remainder below hi's last place, in units of d's last place: r - 2^29 if rounded up
  const int r = (int)((unsigned)b & 0x1fffffffu) - (int)(up << 29);
  const unsigned m = (unsigned)(r < 0 ? -r : r);  // < 2^29
  // m exactly as two floats (each < 2^23, by the 2^23 + k trick), one rounding in the fma
  const float ml = __fsub_rn(__uint_as_float(0x4b000000u | (m & 0x7fffffu)), 8388608.f);
  const float mh = __fsub_rn(__uint_as_float(0x4b000000u | (m >> 23)), 8388608.f);
  const float scale = __uint_as_float((unsigned)(e - 948) << 23);  // 2^(e - 1075)
  const float lo = __fmul_rn(__fmaf_rn(mh, 8388608.f, ml), scale);
  return {hi, ((r < 0) != (sign != 0)) ? -lo : lo};
}

__device__ __forceinline__ F2 df_add_f(F2 a, float b) {
  const F2 s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
// a b + c
__device__ __forceinline__ F2 df_fma(F2 a, F2 b, F2 c) { return df_add(df_mul(a, b), c); }
// 1 / a: the correctly rounded float reciprocal y and the pair y (1 + e + e^2),
// e = 1 - a y (second-order Newton-Raphson step)
__device__ __forceinline__ F2 df_rcp(F2 a) {
  const float y = __frcp_rn(a.hi);
  float e = __fmaf_rn(-a.hi, y, 1.f);
  e = __fmaf_rn(-a.lo, y, e);
  return fast_two_sum(y, __fmul_rn(y, __fmaf_rn(e, e, e)));
}
// sqrt(a), a > 0: the correctly rounded float root and one Newton step on the pair
__device__ __forceinline__ F2 df_sqrt(F2 a) {
  const float s = __fsqrt_rn(a.hi);
  float e = __fmaf_rn(-s, s, a.hi);
  e = __fadd_rn(e, a.lo);
  return fast_two_sum(s, __fmul_rn(e, __fdiv_rn(0.5f, s)));
}

// 1/sqrt(a), a > 0: float estimate y0 (MUFU, ~2^-22), then two Newton-Raphson steps
// y <- y + y (1 - a y^2)/2, the second on the pair (error ~2^-47).
__device__ __forceinline__ F2 df_rsqrt(F2 a) {
  const float y0 = rsqrtf(a.hi);
  // first step in float with the residual formed exactly: e = 1 - a.hi y0^2 - a.lo y0^2
  const float p = __fmul_rn(y0, y0);
  float e = __fmaf_rn(-a.hi, p, 1.f);
  e = __fmaf_rn(-a.hi, __fmaf_rn(y0, y0, -p), e);
  e = __fmaf_rn(-a.lo, p, e);
  const F2 y1 = fast_two_sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), e));
  // second step on pairs
  const F2 r = df_sub(F2{1.f, 0.f}, df_mul(a, df_mul(y1, y1)));
  return df_add(y1, df_mul_f(df_mul(y1, r), 0.5f));
}

// Constant c as a df64 pair, formed at compile time.
struct DFC {
  float hi, lo;
  __host__ __device__ constexpr DFC() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr DFC(double c) : hi((float)c), lo((float)(c - (double)(float)c)) {}
  __device__ __forceinline__ operator F2() const { return {hi, lo}; }
};

// Series coefficients as pairs in the constant bank (the loops over them stay rolled, so
// the per-event code stays small enough for the instruction cache).
static __constant__ DFC kLogSeries[11] = {1.0,      1.0 / 3,  1.0 / 5,  1.0 / 7,
                                          1.0 / 9,  1.0 / 11, 1.0 / 13, 1.0 / 15,
                                          1.0 / 17, 1.0 / 19, 1.0 / 21};  // atanh: 1/(2k+1)
static __constant__ DFC kExpSeries[15] = {1.0,
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
                                          1.0 / 87178291200.0};  // 1/j!

// ---- table-driven exponential and logarithm of a pair ---------------------------------
// Tables of 64 pairs each (filled on the host in FP64, kept in shared memory by the
// kernels that use them): E[j] = 2^(j/64), G[j] = log(1 + (j + 1/2)/64).
constexpr int kTab = 64;

// u = (64 e + j) ln2/64 + r with k = 64 e + j = rint(64 u / ln2), r = u - k C1 - k C23
// (C1 = ln2/64 to 10 bits, so k C1 is exact for |k| < 2^14), |r| <= ln2/128; e^r by its
// Taylor series to r^6/6! (truncation < 1e-19); times E[j] and 2^e (two exact steps).
// Relative error ~1e-15 down to e^u ~ 2^-100, absolute < 2^-149 below; u above 88.5
// gives inf (NaN stays NaN), below -104 gives 0.
__device__ __forceinline__ F2 df_exp_tab(F2 u, const F2* __restrict__ E) {
  if (!(u.hi < 88.5f)) return {u.hi != u.hi ? u.hi : INFINITY, 0.f};
  if (!(u.hi > -104.0f)) return {0.f, 0.f};
  const float k = rintf(__fmul_rn(u.hi, 92.3324826168936563f));  // 64 / ln2
  const float C1 = 0.010833740234375f;                            // 10 significant bits
  constexpr DFC C23(0.0108304246962491474 - 0.010833740234375);
  const F2 r = df_sub(df_add_f(u, -__fmul_rn(k, C1)), df_mul_f(F2(C23), k));
  constexpr DFC c6(1.0 / 720), c5(1.0 / 120), c4(1.0 / 24), c3(1.0 / 6);
  F2 p = df_add(df_mul(F2(c6), r), F2(c5));
  p = df_add(df_mul(p, r), F2(c4));
  p = df_add(df_mul(p, r), F2(c3));
  p = df_add_f(df_mul(p, r), 0.5f);
  p = df_add_f(df_mul(p, r), 1.f);
  p = df_add_f(df_mul(p, r), 1.f);
  const int ki = (int)k;
  const int j = ki & (kTab - 1);
  const int e = (ki - j) / kTab;  // floor(k / 64)
  p = df_mul(p, E[j]);
  const int e1 = e / 2, e2 = e - e1;
  const float s1 = __uint_as_float((unsigned)(e1 + 127) << 23);
  const float s2 = __uint_as_float((unsigned)(e2 + 127) << 23);
  return {__fmul_rn(__fmul_rn(p.hi, s1), s2), __fmul_rn(__fmul_rn(p.lo, s1), s2)};
}

// a = m 2^e, m in [1, 2) from hi's exponent bits (both parts scaled exactly); c = 1 +
// (j + 1/2)/64 from m's top six fraction bits; log m = log c + 2 atanh(s), s = (m - c)/(m + c),
// |s| < 1/256, odd series to s^7 (truncation < 1e-22).  For m >= 3/2 (j >= 32) the pair
// (m/2, c/2) is used instead -- same s -- and e goes up by one, so that log a near 1 has
// no cancellation: G[j] holds log c for j < 32 and log(c/2) for j >= 32.  e ln2 with ln2
// split so that e times its leading part is exact.  Absolute error ~2e-16 plus
// ~1e-15 |log a|.  a outside [2^-100, 2^125) (and a <= 0, NaN) goes to the float logf.
__device__ __forceinline__ F2 df_log_tab(F2 a, const F2* __restrict__ G) {
  if (!(a.hi >= 7.888609052210118e-31f && a.hi < 4.2535295865117308e37f))
    return {logf(a.hi), 0.f};
  const unsigned hb = __float_as_uint(a.hi);
  const int j = (int)((hb >> 17) & 0x3f);
  const int e = (int)((hb >> 23) & 0xff) - 127 + (j >> 5);
  const float sc = __uint_as_float((unsigned)(127 - e) << 23);  // 2^-e, exact
  const F2 m = {__fmul_rn(a.hi, sc), __fmul_rn(a.lo, sc)};
  // c (or c/2), exact in float
  const float c = (1.f + ((float)j + 0.5f) * 0.015625f) * ((j >> 5) ? 0.5f : 1.f);
  const F2 s = df_div(df_add_f(m, -c), df_add_f(m, c));
  const F2 s2 = df_mul(s, s);
  constexpr DFC i7(1.0 / 7), i5(1.0 / 5), i3(1.0 / 3);
  F2 p = df_add(df_mul(F2(i7), s2), F2(i5));
  p = df_add(df_mul(p, s2), F2(i3));
  p = df_add_f(df_mul(p, s2), 1.f);
  const F2 lm = df_add(df_mul(df_mul_f(s, 2.f), p), G[j]);
  if (e == 0) return lm;
  const float L1 = 0.693115234375f;
  constexpr DFC L23(0.69314718055994530942 - 0.693115234375);
  const F2 el = df_add_f(df_mul_f(F2(L23), (float)e), __fmul_rn((float)e, L1));
  return df_add(el, lm);
}

// The tables, one copy per translation unit: filled on the host once per device
// (upload_df_tables, from each unit's kernel preparation), copied into shared memory by
// each block of the kernels that use them (load_df_tables, visible after a barrier).
static __device__ F2 g_exp_tab[kTab], g_log_tab[kTab];
static __shared__ F2 s_exp_tab[kTab], s_log_tab[kTab];

__device__ __forceinline__ void load_df_tables() {
  for (int k = threadIdx.x; k < kTab; k += blockDim.x) {
    s_exp_tab[k] = g_exp_tab[k];
    s_log_tab[k] = g_log_tab[k];
  }
}

static inline cudaError_t upload_df_tables() {
  F2 e[kTab], g[kTab];
  for (int j = 0; j < kTab; ++j) {
    const double ev = std::exp2(j / (double)kTab);
    const double c = 1.0 + (j + 0.5) / kTab;
    const double gv = std::log(j >= kTab / 2 ? 0.5 * c : c);
    e[j].hi = (float)ev;
    e[j].lo = (float)(ev - (double)e[j].hi);
    g[j].hi = (float)gv;
    g[j].lo = (float)(gv - (double)g[j].hi);
  }
  cudaError_t err = cudaMemcpyToSymbol(g_exp_tab, e, sizeof(e));
  if (err == cudaSuccess) err = cudaMemcpyToSymbol(g_log_tab, g, sizeof(g));
  return err;
}

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
  F2 p = kLogSeries[10];
#pragma unroll 1
  for (int k = 9; k >= 0; --k) p = df_add(df_mul(p, s2), kLogSeries[k]);
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
  F2 p = kExpSeries[14];
#pragma unroll 1
  for (int j = 13; j >= 0; --j) p = df_add(df_mul(p, r), kExpSeries[j]);
  const double v = df_to(p);
  return __longlong_as_double(__double_as_longlong(v) + ((long long)k << 52));
}

// ---- value type with operators (template code written for float or double) ----------
// Arithmetic on DF is the pair arithmetic above; values enter from FP64 through from(),
// the bit split (no FP64 conversion instructions), and leave through to_double().
struct DF {
  float hi, lo;
  DF() = default;
  __device__ __forceinline__ constexpr DF(float v) : hi(v), lo(0.f) {}
  __device__ __forceinline__ constexpr DF(F2 v) : hi(v.hi), lo(v.lo) {}
  __device__ __forceinline__ constexpr DF(DFC v) : hi(v.hi), lo(v.lo) {}
  __device__ __forceinline__ operator F2() const { return {hi, lo}; }
  static __device__ __forceinline__ DF from(double v) { return DF(df_split(v)); }
  __device__ __forceinline__ double to_double() const { return df_to(F2{hi, lo}); }
};
__device__ __forceinline__ DF operator+(DF a, DF b) { return df_add(a, b); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return df_sub(a, b); }
__device__ __forceinline__ DF operator-(DF a) { return df_neg(a); }
__device__ __forceinline__ DF operator*(DF a, DF b) { return df_mul(a, b); }
__device__ __forceinline__ DF operator/(DF a, DF b) { return df_div(a, b); }
__device__ __forceinline__ DF& operator+=(DF& a, DF b) { return a = a + b; }
__device__ __forceinline__ bool operator>(DF a, DF b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}

}  // namespace gfi
