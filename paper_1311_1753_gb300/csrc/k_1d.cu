// k_1d.cu -- sm_103a kernels for PDF trees over one or more 1D observables
// (Sec. 2-3 of the paper: per-event evaluate + metric, summed over events).
//
//  k_norm_1d    midpoint-grid normalisation integrals of the Voigtian / threshold leaves
//               (and their parameter derivatives); its last block turns theta and the
//               integrals into per-leaf records (1/N, log N, dlogN, shape constants).
//  k_events_1d  the event stream: SoA columns read with 128-bit loads, the compiled
//               postfix program evaluated per event (forward-mode gradient optional),
//               -log P summed per thread, per block (warp shuffles), and across blocks
//               by the last block in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>
#include "devutil.cuh"
#include "gf_internal.h"
#include "launch.h"
#include "leafrec.h"
#include "sbtab.cuh"

namespace gfi {

// ---- event-side arithmetic ----------------------------------------------------------------
// The per-event program runs in one of two arithmetics with the same code:
//  ArF2  double-float pairs on the FP32 pipe (the normal path: FP64-accurate, no FP64
//        instruction per event except the exact differences x - c of the data and a
//        leaf constant);
//  ArD   plain FP64, for the rare event whose density leaves the float exponent range
//        (P < 2^-80 or > 2^125, or an intermediate that overflows), re-evaluated so that
//        the result is the FP64 one.
struct ArF2 {
  using T = F2;
  static __device__ __forceinline__ T zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ T of(double x) { return df_split(x); }
  static __device__ __forceinline__ T diff(double x, double c) { return df_split(x - c); }
  static __device__ __forceinline__ T add(T a, T b) { return df_add(a, b); }
  static __device__ __forceinline__ T sub(T a, T b) { return df_sub(a, b); }
  static __device__ __forceinline__ T mul(T a, T b) { return df_mul(a, b); }
  static __device__ __forceinline__ T mulf(T a, float b) { return df_mul_f(a, b); }
  static __device__ __forceinline__ T neg(T a) { return df_neg(a); }
  static __device__ __forceinline__ T rcp(T a) { return df_rcp(a); }
  static __device__ __forceinline__ T sqrt_(T a) { return df_sqrt(a); }
  static __device__ __forceinline__ T exp_(T a) { return df_exp_tab(a, s_exp_tab); }
  static __device__ __forceinline__ T log_(T a) { return df_log_tab(a, s_log_tab); }
  static __device__ __forceinline__ bool pos(T a) { return a.hi > 0.f; }
  static __device__ __forceinline__ T two_inv_sqrt_pi() { return DFC(kTwoInvSqrtPi); }
  static __device__ __forceinline__ void faddeeva(T x, T y, const WeidCoef& W, T& wr, T& wi) {
    faddeeva_f2(x, y, W, wr, wi);
  }
};
struct ArD {
  using T = double;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T of(double x) { return x; }
  static __device__ __forceinline__ T diff(double x, double c) { return x - c; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T mulf(T a, float b) { return a * (double)b; }
  static __device__ __forceinline__ T neg(T a) { return -a; }
  static __device__ __forceinline__ T rcp(T a) { return 1.0 / a; }
  static __device__ __forceinline__ T sqrt_(T a) { return sqrt(a); }
  static __device__ __forceinline__ T exp_(T a) { return df_exp(a); }
  static __device__ __forceinline__ T log_(T a) { return df_log(a); }
  static __device__ __forceinline__ bool pos(T a) { return a > 0.0; }
  static __device__ __forceinline__ T two_inv_sqrt_pi() { return kTwoInvSqrtPi; }
  static __device__ __forceinline__ void faddeeva(T x, T y, const WeidCoef& W, T& wr, T& wi) {
    faddeeva_df(x, y, W, wr, wi);
  }
};

// ---- shape functions of the normalisation grid (unnormalised r(x), d r / d local par) ----
// Per-block constants of the leaf's shape, from theta once per block (FP64, then pairs);
// each bin is then evaluated in pairs on the FP32 pipe.
struct ShapeK {
  double x0;        // mu (Voigtian) or x0 (threshold)
  F2 a, b, c, d, e;
  F2 t0, hh;        // grid: lo - x0 and the bin width (midpoint b at t0 + (b + 1/2) hh)
  double rb[10];    // relativistic Breit-Wigner constants (relbw_consts)
  double rb_dm0;    // and its dm0
};

// ---- relativistic Breit-Wigner line shape (Sec. 4: the P-wave D*+ line in the D*+ - D0
// mass difference) ------------------------------------------------------------------------
// f(x) = m Gamma(m) / ((m0^2 - m^2)^2 + m0^2 Gamma(m)^2), m = x + shift, m0 = dm0 + shift,
// Gamma(m) = Gamma0 (q/q0)^{2L+1} (m0/m) B_L(z0)/B_L(z), q^2 = (s - A)(s - B)/(4 s),
// A = (ma + mb)^2, B = (ma - mb)^2, z = q^2 R^2, B_L = 1, 1 + z, 9 + 3 z + z^2; zero at or
// below threshold.  Parameters: dm0, Gamma0, shift, ma, mb, R (the last four fixed).
// s - A is formed as (x - thr)(m + ma + mb), thr = ma + mb - shift, from the exact
// difference x - thr: no cancellation near threshold.
// Constants (the record's c[0..9]): -shift, m0, m0^2, thr, B, R^2,
// k = Gamma0 B_L(z0) m0 / q0^{2L+1} (so Gamma = k q^{2L+1}/(m B_L(z))), 1/Gamma0,
// dln Gamma/dm0 (independent of m), ma + mb.
__device__ inline double rb_poly(int L, double z) {
  return L == 0 ? 1.0 : L == 1 ? 1.0 + z : 9.0 + z * (3.0 + z);
}
__device__ inline void relbw_consts(const LeafDesc& Lf, const double* th, double* c) {
  const double dm0 = th[Lf.par[0]], g0 = th[Lf.par[1]], shift = th[Lf.par[2]];
  const double ma = th[Lf.par[3]], mb = th[Lf.par[4]], R = th[Lf.par[5]];
  const int L = Lf.aux & 0xff;
  const double m0 = dm0 + shift, s0 = m0 * m0;
  const double A = (ma + mb) * (ma + mb), B = (ma - mb) * (ma - mb);
  const double thr = ma + mb - shift;
  const double q02 = (dm0 - thr) * (m0 + ma + mb) * (s0 - B) / (4.0 * s0), z0 = q02 * R * R;
  const double bl0 = rb_poly(L, z0);
  const double dq02 = 2.0 * m0 * (s0 * s0 - A * B) / (4.0 * s0 * s0);  // d q0^2 / d m0
  const double dbl0 = L == 0 ? 0.0 : L == 1 ? 1.0 : 3.0 + 2.0 * z0;
  c[0] = -shift;
  c[1] = m0;
  c[2] = s0;
  c[3] = thr;
  c[4] = B;
  c[5] = R * R;
  c[6] = g0 * bl0 * m0 / pow(q02, L + 0.5);
  c[7] = 1.0 / g0;
  c[8] = -(L + 0.5) * dq02 / q02 + 1.0 / m0 + dbl0 * R * R * dq02 / bl0;
  c[9] = ma + mb;
}
// f and, with G, df/dm0 and df/dGamma0 (unnormalised), in the arithmetic A.  cd: the
// constants in FP64 (x + shift and x - thr enter as exact differences), c: the same in A.
template <class A, bool G>
__device__ __forceinline__ typename A::T relbw_f(double x, const double* cd,
                                                 const typename A::T* c, int L, double pdm0,
                                                 typename A::T& dm0, typename A::T& dg0) {
  using T = typename A::T;
  const T dx = A::diff(x, cd[3]);  // m - ma - mb
  if (!A::pos(dx)) {
    dm0 = dg0 = A::zero();
    return A::zero();
  }
  const T m = A::diff(x, cd[0]);
  const T s = A::mul(m, m);
  const T sa = A::mul(dx, A::add(m, c[9]));  // s - (ma + mb)^2
  const T q2 = A::mul(A::mul(sa, A::sub(s, c[4])), A::rcp(A::mulf(s, 4.f)));
  const T z = A::mul(q2, c[5]);
  const T one = A::of(1.0);
  const T bl = L == 0 ? one
             : L == 1 ? A::add(one, z)
                      : A::add(A::mul(z, A::add(z, A::of(3.0))), A::of(9.0));
  const T sq = A::sqrt_(q2);
  const T qp = L == 0 ? sq : L == 1 ? A::mul(q2, sq) : A::mul(A::mul(q2, q2), sq);
  const T g = A::mul(A::mul(c[6], qp), A::rcp(A::mul(m, bl)));
  const T ds = A::mul(A::neg(A::diff(x, pdm0)), A::add(c[1], m));  // m0^2 - m^2, no cancellation
  const T g2 = A::mul(g, g);
  const T iD = A::rcp(A::add(A::mul(ds, ds), A::mul(c[2], g2)));
  const T f = A::mul(A::mul(m, g), iD);
  if (G) {
    // df/dGamma0 = f/Gamma0 (1 - 2 m0^2 Gamma^2/D)
    dg0 = A::mul(A::mul(f, c[7]), A::sub(one, A::mulf(A::mul(c[2], A::mul(g2, iD)), 2.f)));
    // dGamma = Gamma dlnGamma/dm0;  dD = m0 (4 (m0^2 - m^2) + 2 Gamma^2) + 2 m0^2 Gamma dGamma
    const T dg = A::mul(g, c[8]);
    const T dD = A::add(A::mul(c[1], A::add(A::mulf(ds, 4.f), A::mulf(g2, 2.f))),
                        A::mulf(A::mul(c[2], A::mul(g, dg)), 2.f));
    dm0 = A::mul(A::sub(A::mul(m, dg), A::mul(f, dD)), iD);
  }
  return f;
}

// The grid of a leaf over [lo, hi] relative to x0, in pairs: t0 = lo - x0, hh = (hi - lo)/nbins.
__device__ __forceinline__ void grid_consts(const LeafDesc& L, double x0, ShapeK& K) {
  K.t0 = df_from(L.lo - x0);
  K.hh = df_mul(df_from(L.hi - L.lo), df_rcp(F2{(float)L.nbins, 0.f}));
}

// Voigtian: r = Re w(z)/(sigma sqrt(2 pi)), z = (x - mu)/(sigma sqrt 2) + i Gamma/(2 sigma sqrt 2).
// a = 1/(sigma sqrt2), b = Im z, c = 1/(sigma sqrt(2 pi)), d = 1/sigma, e = a/2: in pairs on
// the FP32 pipe (one thread forms them; FP64 divisions on it would be a long chain).
__device__ __forceinline__ void voigt_consts(double mu, double s, double G, ShapeK& K) {
  const F2 is = df_rcp(df_from(s));
  const F2 a = df_mul(is, F2(DFC(1.0 / kSqrt2)));
  K.x0 = mu;
  K.a = a;
  K.b = df_mul(df_mul_f(df_from(G), 0.5f), a);
  K.c = df_mul(is, F2(DFC(1.0 / kSqrt2Pi)));
  K.d = is;
  K.e = df_mul_f(a, 0.5f);
}
// r and dr/d(mu, sigma, Gamma) at t = x - mu, as pairs (out[0] = r).
__device__ __forceinline__ void voigt_r2(F2 t, const ShapeK& K, const WeidCoef& W, F2* out) {
  const F2 zr = df_mul(t, K.a);
  F2 wr, wi;
  faddeeva_f2(zr, K.b, W, wr, wi);
  const F2 r = df_mul(wr, K.c);
  // w' = -2 z w + 2i/sqrt(pi)
  const F2 dre = df_mul_f(df_sub(df_mul(zr, wr), df_mul(K.b, wi)), -2.f);
  const F2 dim = df_add(df_mul_f(df_add(df_mul(zr, wi), df_mul(K.b, wr)), -2.f),
                        F2(DFC(kTwoInvSqrtPi)));
  out[0] = r;
  out[1] = df_neg(df_mul(df_mul(K.c, K.a), dre));                                 // d/dmu
  out[2] = df_neg(df_add(df_mul(df_mul(K.c, K.d), df_sub(df_mul(dre, zr), df_mul(dim, K.b))),
                         df_mul(r, K.d)));                                           // d/dsigma
  out[3] = df_neg(df_mul(df_mul(K.c, K.e), dim));                                 // d/dGamma
}

// Threshold: r = (x - x0)^p e^{-c (x - x0)} for x > x0.  a = p, b = c.
__device__ __forceinline__ void thresh_consts(double x0, double p, double c, ShapeK& K) {
  K.x0 = x0;
  K.a = df_from(p);
  K.b = df_from(c);
}
// r and dr/d(x0, p, c) at t = x - x0, as pairs.
__device__ __forceinline__ void thresh_r2(F2 T, const ShapeK& K, F2* out) {
  if (!(T.hi > 0.f)) {
    out[0] = out[1] = out[2] = out[3] = F2{0.f, 0.f};
    return;
  }
  const F2 lt = df_log_tab(T, s_log_tab);
  const F2 r = df_exp_tab(df_sub(df_mul(K.a, lt), df_mul(K.b, T)), s_exp_tab);
  out[0] = r;
  out[1] = df_mul(r, df_sub(K.b, df_mul(K.a, df_rcp(T))));
  out[2] = df_mul(r, lt);
  out[3] = df_neg(df_mul(T, r));
}

// ---- leaf records ------------------------------------------------------------------------
// rec[0] = 1/N, rec[1] = log N, rec[2 + k] = d log N / d par_k, rec[10 + j] = constants.
// A leaf flagged kRawLeaf (the core and shell of a CompositePdf) keeps its unnormalised
// shape: N = 1 and dN = 0.
__device__ __noinline__ void make_leaf_record(const LeafDesc& L, const double* th, double N, const double* dN,
                                 double* rec) {
  for (int k = 0; k < kLeafRec; ++k) rec[k] = 0.0;
  const double lo = L.lo, hi = L.hi;
  double* c = rec + 10;
  const bool raw = (L.aux & kRawLeaf) != 0;
  const double zero3[3] = {0.0, 0.0, 0.0};
  if (raw) {
    N = 1.0;
    dN = zero3;
  }
  switch (L.kind) {
    case L_EXP:
    case L_GAUSS:
      analytic_leaf_record(L, th, raw, rec);  // leafrec.h (also computed on the host)
      break;
    case L_VOIGT: {
      // two FP64 reciprocals (GB300's FP64 divisions are long serial sequences)
      const double mu = th[L.par[0]], s = th[L.par[1]], G = th[L.par[2]];
      const double iN = 1.0 / N, is = 1.0 / s;
      rec[0] = iN;
      rec[1] = log(N);
      for (int k = 0; k < 3; ++k) rec[2 + k] = dN[k] * iN;
      c[0] = mu;
      c[1] = is * (1.0 / kSqrt2);
      c[2] = 0.5 * G * c[1];
      c[3] = is * iN * (1.0 / kSqrt2Pi);
      c[4] = is;
      // products the event-side gradient uses
      c[5] = c[3] * c[1];
      c[6] = c[3] * c[4];
      c[7] = 0.5 * c[3] * c[1];
      c[8] = c[4] + rec[3];
      break;
    }
    case L_THRESH: {
      const double iN = 1.0 / N;
      rec[0] = iN;
      rec[1] = log(N);
      for (int k = 0; k < 3; ++k) rec[2 + k] = dN[k] * iN;
      c[0] = th[L.par[0]];
      c[1] = th[L.par[1]];
      c[2] = th[L.par[2]];
      c[3] = iN;
      break;
    }
    case L_RELBW: {
      rec[0] = 1.0 / N;
      rec[1] = log(N);
      rec[2] = dN[0] / N;
      rec[3] = dN[1] / N;
      rec[4] = L.aux & 0xff;   // orbital angular momentum and dm0 (the other dlogN slots
      rec[5] = th[L.par[0]];   // are unused)
      relbw_consts(L, th, c);
      break;
    }
    case L_CONV:
    case L_GNORM:
      break;  // written after this kernel (k_conv_sum, k_gnorm)
    case L_IND: {
      // [c0, c1) with c0, c1 the boundary parameters (aux bit 1: lower, bit 2: upper) or
      // the range ends; the interval reaching hi is closed (c1 = +inf)
      rec[0] = 1.0;
      c[0] = (L.aux & 1) ? th[L.par[0]] : -INFINITY;
      c[1] = (L.aux & 2) ? th[L.par[(L.aux & 1) ? 1 : 0]] : INFINITY;
      break;
    }
    case L_POLY: {
      // N = Q(hi) - Q(lo), Q(x) = sum_k a_k x^{k+1}/(k+1)
      double n = 0.0, phk = hi, plk = lo;
      double ik[kMaxLocal];
      for (int k = 0; k < L.npar; ++k) {
        ik[k] = raw ? 0.0 : (phk - plk) / (k + 1);
        n = fma(th[L.par[k]], ik[k], n);
        phk *= hi;
        plk *= lo;
      }
      if (raw) n = 1.0;
      rec[0] = 1.0 / n;
      rec[1] = log(n);
      for (int k = 0; k < L.npar; ++k) {
        rec[2 + k] = ik[k] / n;
        c[k] = th[L.par[k]] / n;
      }
      break;
    }
  }
}

__device__ inline void make_coefs(const Program& P, const double* th, double* coef) {
  for (int j = 0; j < P.ncoef; ++j) {
    const CoefDesc& C = P.coef[j];
    if (C.sign > 0) {
      coef[j] = th[C.par[0]];
    } else {
      double s = 1.0;
      for (int k = 0; k < C.n; ++k) s -= th[C.par[k]];
      coef[j] = s;
    }
  }
}

// The Voigtian's and the threshold's leaf records from the pair sums S = (N, dN/dpar_k)
// of their grids, formed in pairs on the FP32 pipe by a whole warp: every lane takes the
// same steps, then lane k converts value k to FP64 and stores it (one conversion per lane
// instead of a chain of FP64 divisions, logarithm and conversions on one thread).  The
// parameters the events subtract (mu, x0) and the threshold's (p, c) are copied exactly.
// Same layout as make_leaf_record.
__device__ __forceinline__ void leaf_record_warp(const LeafDesc& L, const double* th,
                                                 const F2* S, double* rec) {
  const int lane = threadIdx.x & 31;
  const bool raw = (L.aux & kRawLeaf) != 0;
  const F2 z = {0.f, 0.f};
  const F2 N = raw ? F2{1.f, 0.f} : S[0];
  const F2 iN = df_rcp(N);
  const F2 lN = raw ? z : df_log_tab(N, s_log_tab);
  const F2 r2 = raw ? z : df_mul(S[1], iN), r3 = raw ? z : df_mul(S[2], iN),
           r4 = raw ? z : df_mul(S[3], iN);
  F2 v = z;
  bool exact = false;  // this lane copies a parameter
  if (lane == 0) v = iN;
  if (lane == 1) v = lN;
  if (lane == 2) v = r2;
  if (lane == 3) v = r3;
  if (lane == 4) v = r4;
  if (L.kind == L_VOIGT) {
    const F2 is = df_rcp(df_from(th[L.par[1]]));
    const F2 c1 = df_mul(is, F2(DFC(1.0 / kSqrt2)));
    const F2 c3 = df_mul(df_mul(is, iN), F2(DFC(1.0 / kSqrt2Pi)));
    const F2 c31 = df_mul(c3, c1);
    exact = lane == 10;  // mu
    if (lane == 11) v = c1;
    if (lane == 12) v = df_mul(df_mul_f(df_from(th[L.par[2]]), 0.5f), c1);
    if (lane == 13) v = c3;
    if (lane == 14) v = is;
    if (lane == 15) v = c31;
    if (lane == 16) v = df_mul(c3, is);
    if (lane == 17) v = df_mul_f(c31, 0.5f);
    if (lane == 18) v = df_add(is, r3);
  } else {  // L_THRESH: x0, p, c, then 1/N
    exact = lane >= 10 && lane < 13;
    if (lane == 13) v = iN;
  }
  if (lane < kLeafRec) rec[lane] = exact ? th[L.par[lane - 10]] : df_to(v);
}

// ---- normalisation grid -----------------------------------------------------------------
// One block per (grid leaf, chunk of kThreads bins): each thread takes one midpoint.
// partials (value-major within a block): [block][4] = (sum r, sum dr/dp0, dr/dp1, dr/dp2).
// Body of one (virtual) block vb of the vgrid blocks of a normalisation launch; the last
// block to arrive finishes.  Shared scratch: red[32], *last, sums[kMaxLeaf][4] (pairs).
// The Voigtian and threshold grids run in pairs end to end (bin positions, values, block
// and cross-block sums, records); other leaves evaluate in FP64 and enter the pair sums.
__device__ __forceinline__ void norm_1d_block(const Program& P, const WeidCoef& W,
                                              const double* __restrict__ theta,
                                              double* __restrict__ partials,
                                              unsigned* __restrict__ counter,
                                              double* __restrict__ derived, int vb, int vgrid,
                                              double* red, int* last, F2 (*sums)[4],
                                              ShapeK* shk) {
  // locate this block's leaf
  int li = -1;
  for (int l = 0; l < P.nleaf; ++l) {
    const LeafDesc& L = P.leaf[l];
    if (L.nbins > 0 && vb >= L.grid_first_block && vb < L.grid_first_block + L.grid_nblocks)
      li = l;
  }
  if (li >= 0 && threadIdx.x == 0) {
    const LeafDesc& L = P.leaf[li];
    if (L.kind == L_VOIGT) {
      voigt_consts(theta[L.par[0]], theta[L.par[1]], theta[L.par[2]], *shk);
      grid_consts(L, shk->x0, *shk);
    } else if (L.kind == L_RELBW) {
      relbw_consts(L, theta, shk->rb);
      shk->rb_dm0 = theta[L.par[0]];
    } else {
      thresh_consts(theta[L.par[0]], theta[L.par[1]], theta[L.par[2]], *shk);
      grid_consts(L, shk->x0, *shk);
    }
  }
  __syncthreads();
  F2 v[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  if (li >= 0) {
    const LeafDesc& L = P.leaf[li];
    const int b = (vb - L.grid_first_block) * blockDim.x + threadIdx.x;
    if (b < L.nbins) {
      if (L.kind == L_RELBW) {
        const double h = (L.hi - L.lo) / L.nbins;
        const double x = L.lo + (b + 0.5) * h;
        double d0, d1;
        v[0] = df_from(relbw_f<ArD, true>(x, shk->rb, shk->rb, L.aux & 0xff, shk->rb_dm0, d0, d1));
        v[1] = df_from(d0);
        v[2] = df_from(d1);
      } else {
        const F2 t = df_add(shk->t0, df_mul_f(shk->hh, (float)b + 0.5f));
        if (L.kind == L_VOIGT) voigt_r2(t, *shk, W, v);
        else thresh_r2(t, *shk, v);
      }
    }
  }
  // the four block sums in one pass (pairs, their shuffle trees interleaved)
  block_sum_pairs<4>([&](int k) -> F2 { return v[k]; }, 4, red, partials + (size_t)vb * 4);
  if (!arrive_last_of(counter, (unsigned)vgrid, last)) return;
  // last block: one warp per (leaf, value), its lanes' loads of the leaf's chunk partials
  // all in flight, fixed-order pair sums times the bin width; then every leaf record
  {
    constexpr int kPer = 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = warp; q < 4 * P.nleaf; q += nw) {
      const LeafDesc& L = P.leaf[q >> 2];
      const int k = q & 3;
      if (L.nbins <= 0) continue;  // uniform over the warp
      F2 a = {0.f, 0.f};
      for (int b0 = 0; b0 < L.grid_nblocks; b0 += 32 * kPer) {
        double t[kPer];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
          const int b = b0 + lane + 32 * j;
          t[j] = b < L.grid_nblocks ? __ldcg(partials + (size_t)(L.grid_first_block + b) * 4 + k)
                                    : 0.0;
        }
#pragma unroll
        for (int j = 0; j < kPer; ++j)  // the padding skipped (df_split's zero path is a call)
          if (b0 + lane + 32 * j < L.grid_nblocks) a = df_add(a, df_split(t[j]));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const F2 u = {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
        a = df_add(a, u);
      }
      if (lane == 0)
        sums[q >> 2][k] = df_mul(a, df_mul(df_from(L.hi - L.lo), df_rcp(F2{(float)L.nbins, 0.f})));
    }
  }
  __syncthreads();
  // one leaf per warp: the Voigtian's and threshold's records by the whole warp in pairs,
  // the others by its lane 0 in FP64 (the leaves' records side by side, not as divergent
  // branches of one warp)
  {
    const int lane = threadIdx.x & 31;
    for (int l = threadIdx.x >> 5; l < P.nleaf; l += blockDim.x >> 5) {
      const LeafDesc& L = P.leaf[l];
      if (L.nbins > 0 && (L.kind == L_VOIGT || L.kind == L_THRESH)) {
        leaf_record_warp(L, theta, sums[l], derived + l * kLeafRec);
      } else if (lane == 0) {
        const double dN[3] = {df_to(sums[l][1]), df_to(sums[l][2]), df_to(sums[l][3])};
        make_leaf_record(L, theta, df_to(sums[l][0]), dN, derived + l * kLeafRec);
      }
    }
  }
  if (threadIdx.x == 0) {
    make_coefs(P, theta, derived + kMaxLeaf * kLeafRec);
    *counter = 0u;
  }
}

// Copy the program into shared memory (every block, before its first use).
__device__ __forceinline__ void load_program(const Program* __restrict__ src, Program& dst) {
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(&dst);
  for (int k = threadIdx.x; k < (int)(sizeof(Program) / 4); k += blockDim.x) d[k] = __ldg(s + k);
  __syncthreads();
}

// The normalisation launch: blocks 0 .. nnorm - 1 the grids, the rest (if tab) the entries
// of the signal + background kernel's table of w expansions (independent of the grids).
__global__ void __launch_bounds__(kThreads) k_norm_1d(const Program* __restrict__ Pg,
                                                      const __grid_constant__ WeidCoef W,
                                                      const double* __restrict__ theta,
                                                      double* __restrict__ partials,
                                                      unsigned* __restrict__ counter,
                                                      double* __restrict__ derived, int nnorm,
                                                      const SBTabHdr* __restrict__ hdr,
                                                      float4* __restrict__ tab) {
  if ((int)blockIdx.x >= nnorm) {
    const int nt = ((int)gridDim.x - nnorm) * blockDim.x;
    const int ntab = hdr->ntab;
    for (int j = ((int)blockIdx.x - nnorm) * blockDim.x + threadIdx.x; j < ntab; j += nt)
      sbtab_build(j, *hdr, W, tab);
    return;
  }
  __shared__ Program P;
  __shared__ double red[32];
  __shared__ int last;
  __shared__ F2 sums[kMaxLeaf][4];
  __shared__ ShapeK shk;
  load_df_tables();
  load_program(Pg, P);
  norm_1d_block(P, W, theta, partials, counter, derived, blockIdx.x, nnorm, red, &last, sums,
                &shk);
}

// ---- per-chunk expansion of w(z) on sorted data ------------------------------------------
// With the events sorted by the Voigtian's observable, a thread's chunk of kChunk
// consecutive events spans a short interval of z = (x - mu)/(sigma sqrt2) + i y.  The
// thread evaluates w exactly at the chunk's middle event z0 (faddeeva_f2) and builds the
// Taylor coefficients t_k = w^(k)(z0)/k! from the differential equation w' = -2 z w +
// 2i/sqrt(pi):  t_1 = -2 z0 t_0 + 2i/sqrt(pi),  t_{k+1} = -2 (z0 t_k + t_{k-1})/(k + 1).
// Each event then takes w(z0 + d) = sum_k t_k d^k, d = Re z - Re z0 real, to degree
// kTayDeg.  Used only when the chunk's largest |d| is at most kTayLim: |t_k| <= 3 on the
// unit circle around any z0 with Im z0 >= 0 (Cauchy), so the truncation is below
// 3 kTayLim^6 ~ 2e-21, and the coefficient rounding (amplified ~2|z0|^2 by the
// recurrence at large |z0|) adds < 2e-13 relative to Re w at |z0| = 37, below the
// series' own error there.  Wider chunks evaluate w directly per event.
constexpr int kTayDeg = 5;
constexpr float kTayLim = 3e-4f;

struct Tay {
  int slot;   // leaf record of the expanded Voigtian leaf, -1: none
  bool ok;    // the current chunk uses the expansion
  F2 z0;      // Re z0 (Im z0 is the leaf constant c[2])
  F2* t;      // shared memory: t_k as (re, im) pairs, [kTayDeg + 1][2][stride], this thread
  int stride;
};

__device__ __forceinline__ void cmul2(F2 ar, F2 ai, F2 br, F2 bi, F2& cr, F2& ci) {
  cr = df_sub(df_mul(ar, br), df_mul(ai, bi));
  ci = df_add(df_mul(ar, bi), df_mul(ai, br));
}

// Expansion of w at z0 = zr + i y into tay.t (caller checked the chunk width).
__device__ __forceinline__ void tay_build(Tay& tay, F2 zr, F2 y, const WeidCoef& W) {
  F2 tr[kTayDeg + 1], ti[kTayDeg + 1];
  faddeeva_f2(zr, y, W, tr[0], ti[0]);
  F2 ar, ai;
  cmul2(zr, y, tr[0], ti[0], ar, ai);  // z0 t0
  tr[1] = df_mul_f(ar, -2.f);
  ti[1] = df_add(df_mul_f(ai, -2.f), DFC(kTwoInvSqrtPi));
  constexpr DFC sc[kTayDeg] = {0.0, 1.0, 2.0 / 3, 0.5, 2.0 / 5};  // 2/(k + 1), k >= 1
#pragma unroll
  for (int k = 1; k < kTayDeg; ++k) {
    cmul2(zr, y, tr[k], ti[k], ar, ai);
    const F2 s = F2(sc[k]);
    tr[k + 1] = df_neg(df_mul(df_add(ar, tr[k - 1]), s));
    ti[k + 1] = df_neg(df_mul(df_add(ai, ti[k - 1]), s));
  }
#pragma unroll
  for (int k = 0; k <= kTayDeg; ++k) {
    tay.t[(2 * k) * tay.stride] = tr[k];
    tay.t[(2 * k + 1) * tay.stride] = ti[k];
  }
  tay.z0 = zr;
}

__device__ __forceinline__ void tay_eval(const Tay& tay, F2 zr, F2& wr, F2& wi) {
  const F2 d = df_sub(zr, tay.z0);
  wr = tay.t[(2 * kTayDeg) * tay.stride];
  wi = tay.t[(2 * kTayDeg + 1) * tay.stride];
#pragma unroll
  for (int k = kTayDeg - 1; k >= 0; --k) {
    wr = df_add(df_mul(wr, d), tay.t[(2 * k) * tay.stride]);
    wi = df_add(df_mul(wi, d), tay.t[(2 * k + 1) * tay.stride]);
  }
}

// ---- event-side leaf evaluation ------------------------------------------------------------
// Returns the normalised leaf value (log domain for EXP and GAUSS).  With G, adds the
// partials with respect to the leaf's free parameters into the gradient slot g (stride bd).
// rec: the leaf record in FP64 (its constant c0 = rec[10] enters the exact difference
// x - c0); r: the same record in the arithmetic A.
// EXT: also the line shape, convolution and indicator leaves (false in the AddPdf-of-leaves
// path, which the compiler gives the basic leaves only).
template <class A, bool G, bool EXT = true, class Sink>
__device__ __forceinline__ typename A::T eval_leaf_s(const Instr& I, const double* rec,
                                                     const typename A::T* r, double x,
                                                     const WeidCoef& W, Sink sink,
                                                     const Tay* tay) {
  using T = typename A::T;
  const T* c = r + 10;
  switch (I.kind) {
    case L_EXP: {
      const T X = A::of(x);
      if (G && I.gidx[0] >= 0) sink(0, A::sub(X, r[2]));
      return A::add(A::mul(c[0], X), c[1]);
    }
    case L_GAUSS: {
      const T u = A::mul(A::diff(x, rec[10]), c[1]);
      if (G) {
        const T uc = A::mul(u, c[1]);
        if (I.gidx[0] >= 0) sink(0, A::sub(uc, r[2]));
        if (I.gidx[1] >= 0)
          sink(1, A::sub(A::mul(u, uc), r[3]));
      }
      return A::add(A::mulf(A::mul(u, u), -0.5f), c[2]);
    }
    case L_VOIGT: {
      const T zr = A::mul(A::diff(x, rec[10]), c[1]);
      T wr, wi;
      if constexpr (std::is_same<A, ArF2>::value) {
        if (tay && tay->ok && I.slot == tay->slot) tay_eval(*tay, zr, wr, wi);
        else A::faddeeva(zr, c[2], W, wr, wi);
      } else {
        A::faddeeva(zr, c[2], W, wr, wi);
      }
      const T l = A::mul(c[3], wr);
      if (G) {
        // w' = -2 z w + 2i/sqrt(pi)
        const T dre = A::mulf(A::sub(A::mul(zr, wr), A::mul(c[2], wi)), -2.f);
        const T dim = A::add(A::mulf(A::add(A::mul(zr, wi), A::mul(c[2], wr)), -2.f),
                             A::two_inv_sqrt_pi());
        if (I.gidx[0] >= 0)
          sink(0, A::neg(A::add(A::mul(c[5], dre), A::mul(l, r[2]))));
        if (I.gidx[1] >= 0) {
          const T q = A::sub(A::mul(dre, zr), A::mul(dim, c[2]));
          sink(1, A::neg(A::add(A::mul(c[6], q), A::mul(l, c[8]))));
        }
        if (I.gidx[2] >= 0)
          sink(2, A::neg(A::add(A::mul(c[7], dim), A::mul(l, r[4]))));
      }
      return l;
    }
    case L_THRESH: {
      const T t = A::diff(x, rec[10]);
      if (!A::pos(t)) return A::zero();
      T l, lt = A::zero();
      if (rec[11] == 0.5 && !(G && I.gidx[1] >= 0)) {
        l = A::mul(A::mul(A::sqrt_(t), A::exp_(A::neg(A::mul(c[2], t)))), c[3]);
      } else {
        lt = A::log_(t);
        l = A::mul(A::exp_(A::sub(A::mul(c[1], lt), A::mul(c[2], t))), c[3]);
      }
      if (G) {
        if (I.gidx[0] >= 0)
          sink(0, A::mul(l, A::sub(A::sub(c[2], A::mul(c[1], A::rcp(t))), r[2])));
        if (I.gidx[1] >= 0)
          sink(1, A::mul(l, A::sub(lt, r[3])));
        if (I.gidx[2] >= 0)
          sink(2, A::neg(A::mul(l, A::add(t, r[4]))));
      }
      return l;
    }
    case L_RELBW: {
      if constexpr (!EXT) return A::zero();
      T dm, dg;
      const T f = relbw_f<A, G>(x, rec + 10, c, (int)rec[4], rec[5], dm, dg);
      const T l = A::mul(f, r[0]);
      if (G) {
        if (I.gidx[0] >= 0) sink(0, A::sub(A::mul(dm, r[0]), A::mul(l, r[2])));
        if (I.gidx[1] >= 0) sink(1, A::sub(A::mul(dg, r[0]), A::mul(l, r[3])));
      }
      return l;
    }
    case L_IND:
      if constexpr (!EXT) return A::zero();
      return (x >= rec[10] && x < rec[11]) ? A::of(1.0) : A::zero();
    case L_CONV: {
      if constexpr (!EXT) return A::zero();
      // lattice table (k_conv_sum): C_i then dC_i/dtheta_l, rows of L + 1; linear in
      // between (FP64 index arithmetic: convolutions serve binned or modest data)
      const double* T_ = reinterpret_cast<const double*>(__double_as_longlong(rec[13]));
      const int Lt = (int)rec[12];
      const double sd = (x - rec[10]) * rec[11];
      int k = (int)floor(sd);
      k = k < 0 ? 0 : (k > Lt - 1 ? Lt - 1 : k);
      const double u = sd - k;
      const T l = A::mul(A::of(fma(u, T_[k + 1] - T_[k], T_[k])), r[0]);
      if (G)
        for (int j = 0; j < I.npar; ++j)
          if (I.gidx[j] >= 0) {
            const double* Tj = T_ + (size_t)(1 + j) * (Lt + 1);
            sink(j, A::sub(A::mul(A::of(fma(u, Tj[k + 1] - Tj[k], Tj[k])), r[0]),
                           A::mul(l, r[2 + j])));
          }
      return l;
    }
    case L_POLY: {
      const T X = A::of(x);
      T l = A::zero();
      for (int k = I.npar - 1; k >= 0; --k) l = A::add(A::mul(l, X), c[k]);
      if (G) {
        T xk = r[0];
        for (int k = 0; k < I.npar; ++k) {
          if (I.gidx[k] >= 0)
            sink(k, A::sub(xk, A::mul(l, r[2 + k])));
          xk = A::mul(xk, X);
        }
      }
      return l;
    }
  }
  return A::zero();
}

template <class A, bool G>
__device__ __forceinline__ typename A::T eval_leaf(const Instr& I, const double* rec,
                                                   const typename A::T* r, double x,
                                                   const WeidCoef& W, typename A::T* g,
                                                   int bd, const Tay* tay) {
  using T = typename A::T;
  return eval_leaf_s<A, G>(I, rec, r, x, W,
                           [&](int j, T term) { g[I.gidx[j] * bd] = A::add(g[I.gidx[j] * bd], term); },
                           tay);
}

// Shell of a CompositePdf (Sec. 3) at u: its unnormalised shape f(u), f'(u) and, with G,
// df/d(local parameter j) into dp[j].  Constants c: EXP a; GAUSS mu, 1/sigma; POLY a_k
// (the leaf's record with kRawLeaf: N = 1).
template <class A, bool G>
__device__ __forceinline__ void shell_f(int kind, int npar, const typename A::T* c,
                                        typename A::T u, typename A::T& f, typename A::T& fu,
                                        typename A::T* dp) {
  using T = typename A::T;
  if (kind == L_EXP) {
    f = A::exp_(A::mul(c[0], u));
    fu = A::mul(c[0], f);
    if (G) dp[0] = A::mul(u, f);
  } else if (kind == L_GAUSS) {
    const T t = A::mul(A::sub(u, c[0]), c[1]);
    f = A::exp_(A::mulf(A::mul(t, t), -0.5f));
    const T tf = A::mul(A::mul(t, f), c[1]);  // t f / sigma
    fu = A::neg(tf);
    if (G) {
      dp[0] = tf;
      dp[1] = A::mul(t, tf);
    }
  } else {  // L_POLY: Horner for f and f'
    f = c[npar - 1];
    fu = A::zero();
    for (int k = npar - 2; k >= 0; --k) {
      fu = A::add(A::mul(fu, u), f);
      f = A::add(A::mul(f, u), c[k]);
    }
    if (G) {
      T uk = A::of(1.0);
      for (int k = 0; k < npar; ++k) {
        dp[k] = uk;
        uk = A::mul(uk, u);
      }
    }
  }
}

// The compiled postfix program for one event: returns the root's value (log domain if
// P.root_log) and, with G, leaves its gradient in stack level 0 of dyn (stride bd).
template <class A, bool G>
__device__ __forceinline__ typename A::T run_program(const Program& P, const double* rec,
                                                     const typename A::T* rc, const double* x,
                                                     const WeidCoef& W, typename A::T* dyn,
                                                     int nf, int bd, int tid,
                                                     const Tay* tay = nullptr) {
  using T = typename A::T;
  const T* coef = rc + kMaxLeaf * kLeafRec;
  T s0 = A::zero(), s1 = A::zero(), s2 = A::zero(), s3 = A::zero();
  int dep = 0;
  for (int pc = 0; pc < P.n; ++pc) {
    const Instr& I = P.ins[pc];
    T* gt = dyn + (size_t)(dep - 1) * nf * bd + tid;  // gradient of s0
    switch (I.op) {
      case OP_LEAF: {
        T* gn = dyn + (size_t)dep * nf * bd + tid;
        if (G)
          for (int k = 0; k < nf; ++k) gn[k * bd] = A::zero();
        const T v = eval_leaf<A, G>(I, rec + I.slot * kLeafRec, rc + I.slot * kLeafRec, x[I.obs],
                                    W, gn, bd, tay);
        s3 = s2; s2 = s1; s1 = s0; s0 = v;
        ++dep;
        break;
      }
      case OP_TOLIN: {
        s0 = A::exp_(s0);
        if (G)
          for (int k = 0; k < nf; ++k) gt[k * bd] = A::mul(gt[k * bd], s0);
        break;
      }
      case OP_MUL: {
        if (G) {
          T* gb = gt - (size_t)nf * bd;
          for (int k = 0; k < nf; ++k)
            gb[k * bd] = A::add(A::mul(gb[k * bd], s0), A::mul(gt[k * bd], s1));
        }
        s0 = A::mul(s1, s0); s1 = s2; s2 = s3;
        --dep;
        break;
      }
      case OP_LMUL:
      case OP_ADD: {
        if (G) {
          T* gb = gt - (size_t)nf * bd;
          for (int k = 0; k < nf; ++k) gb[k * bd] = A::add(gb[k * bd], gt[k * bd]);
        }
        s0 = A::add(s1, s0); s1 = s2; s2 = s3;
        --dep;
        break;
      }
      case OP_COMPOSE: {
        // shell(u), u = s0 (the core's value): d/dtheta = f'(u) du/dtheta + df/dtheta_shell
        const T* c = rc + I.slot * kLeafRec + 10;
        T f, fu, dp[kMaxLocal];
        shell_f<A, G>(I.kind, I.npar, c, s0, f, fu, dp);
        if (G) {
          for (int k = 0; k < nf; ++k) gt[k * bd] = A::mul(gt[k * bd], fu);
          for (int j = 0; j < I.npar; ++j)
            if (I.gidx[j] >= 0) gt[I.gidx[j] * bd] = A::add(gt[I.gidx[j] * bd], dp[j]);
        }
        s0 = f;
        break;
      }
      case OP_GNORM: {
        // s0 / N: d/dtheta = ds0/N - (s0/N) dlogN/dtheta (the node's local parameters)
        const T* r = rc + I.slot * kLeafRec;
        s0 = A::mul(s0, r[0]);
        if (G) {
          for (int k = 0; k < nf; ++k) gt[k * bd] = A::mul(gt[k * bd], r[0]);
          for (int j = 0; j < I.npar; ++j)
            if (I.gidx[j] >= 0)
              gt[I.gidx[j] * bd] = A::sub(gt[I.gidx[j] * bd], A::mul(s0, r[2 + j]));
        }
        break;
      }
      case OP_SCALE: {
        const T cf = coef[I.slot];
        if (G) {
          for (int k = 0; k < nf; ++k) gt[k * bd] = A::mul(gt[k * bd], cf);
          for (int j = 0; j < I.npar; ++j)
            if (I.gidx[j] >= 0)
              gt[I.gidx[j] * bd] = A::add(gt[I.gidx[j] * bd], A::mulf(s0, (float)I.kind));
        }
        s0 = A::mul(s0, cf);
        break;
      }
    }
  }
  return s0;
}

// The FP64 re-evaluation, out of line: it is rarely taken and keeps its code out of the
// hot loop's instruction stream.
template <bool G>
__device__ __noinline__ double run_program_fp64(const Program& P, const double* rec,
                                                const double* x, const WeidCoef& W, double* dyn,
                                                int nf, int bd, int tid) {
  return run_program<ArD, G>(P, rec, rec, x, W, dyn, nf, bd, tid);
}

// AddPdf of leaves (P.mix = K components) for one event: P = sum_k c_k L_k, each leaf by
// the same code as the interpreter's.  With G, the thread's slots comp[(4k + e) bd] get
// L_k (e = 0) and dL_k/d(local parameter e - 1) (e = 1..3, linear domain); the caller adds
// c_k dL_k/P and +-L_k/P into the gradient sums once P is known.
template <bool G>
__device__ __forceinline__ F2 run_mixture(const Program& P, const double* rec, const F2* rf,
                                          const double* x, const WeidCoef& W, F2* comp, int bd,
                                          const Tay* tay) {
  const F2* coef = rf + kMaxLeaf * kLeafRec;
  F2 s = {0.f, 0.f};
  for (int k = 0; k < P.mix; ++k) {
    const Instr& I = P.ins[P.mix_leaf[k]];
    F2 d0 = {0.f, 0.f}, d1 = {0.f, 0.f}, d2 = {0.f, 0.f};
    F2 v = eval_leaf_s<ArF2, G, false>(
        I, rec + I.slot * kLeafRec, rf + I.slot * kLeafRec, x[I.obs], W,
        [&](int j, F2 t) {
          if (j == 0) d0 = t;
          else if (j == 1) d1 = t;
          else d2 = t;
        },
        tay);
    if (P.mix_log[k]) {  // log-domain leaf: L = e^v, dL = L dv
      v = df_exp_tab(v, s_exp_tab);
      if (G) {
        d0 = df_mul(d0, v);
        d1 = df_mul(d1, v);
        d2 = df_mul(d2, v);
      }
    }
    if (G) {
      comp[(4 * k) * bd] = v;
      comp[(4 * k + 1) * bd] = d0;
      comp[(4 * k + 2) * bd] = d1;
      comp[(4 * k + 3) * bd] = d2;
    }
    const F2 t = df_mul(v, coef[P.ins[P.mix_scale[k]].slot]);
    s = k == 0 ? t : df_add(s, t);
  }
  return s;
}

// Gradient sums of one mixture event: sc = -1/P.
__device__ __forceinline__ void mixture_grad(const Program& P, const F2* rf, const F2* comp,
                                             F2 sc, F2* gacc, int bd) {
  const F2* coef = rf + kMaxLeaf * kLeafRec;
  for (int k = 0; k < P.mix; ++k) {
    const Instr& I = P.ins[P.mix_leaf[k]];
    const Instr& S = P.ins[P.mix_scale[k]];
    const F2 cs = df_mul(coef[S.slot], sc);
#pragma unroll
    for (int j = 0; j < kMixLocal; ++j)
      if (j < I.npar && I.gidx[j] >= 0) {
        F2& g = gacc[I.gidx[j] * bd];
        g = df_add(g, df_mul(comp[(4 * k + 1 + j) * bd], cs));
      }
    const F2 vs = df_mul(comp[(4 * k) * bd], sc);
    for (int q = 0; q < S.npar; ++q)
      if (S.gidx[q] >= 0) {
        F2& g = gacc[S.gidx[q] * bd];
        g = df_add(g, S.kind > 0 ? vs : df_neg(vs));
      }
  }
}

// ---- binned metrics ------------------------------------------------------------------------
// One bin (Sec. 2: the metric applied to the PDF's value at the bin centre): contents n,
// expected nu = K P.  term: the bin's share of the metric; dP: the factor of the
// gradient's dP/dtheta (linear root) or, for a log-domain root, of dlogP/dtheta (dlog).
//   NLL (multinomial)  -n log P             dP = -n / P          dlog = -n
//   BINNED_NLL         nu - n log nu        dP = K - n / P       dlog = nu - n
//   CHISQ              (n - nu)^2 / s2      dP = -2 (n - nu) K/s2  dlog = -2 (n - nu) nu/s2
// In pairs, for P in the float range (P > 0).
__device__ __forceinline__ void bin_metric_f2(const Program& P, int64_t i, F2 lp, F2 pv, F2 kb,
                                              F2 lk, F2& term, F2& fac) {
  const double nd = P.bw[i];
  const F2 n = df_split(nd);
  const bool lin = !P.root_log;
  if (P.metric == 0) {
    term = nd == 0.0 ? F2{0.f, 0.f} : df_neg(df_mul(n, lp));
    fac = lin ? (nd == 0.0 ? F2{0.f, 0.f} : df_neg(df_mul(n, df_rcp(pv)))) : df_neg(n);
    return;
  }
  const F2 nu = df_mul(kb, pv);
  if (P.metric == 1) {
    term = nd == 0.0 ? nu : df_sub(nu, df_mul(n, df_add(lp, lk)));
    fac = lin ? (nd == 0.0 ? kb : df_sub(kb, df_mul(n, df_rcp(pv)))) : df_sub(nu, n);
    return;
  }
  const F2 is2 = df_rcp(df_split(P.bs2[i]));
  const F2 r = df_sub(n, nu);
  term = df_mul(df_mul(r, r), is2);
  fac = df_mul_f(df_mul(df_mul(r, lin ? kb : nu), is2), -2.f);
}
// The same in FP64 for the re-evaluated bins (P may be 0 or outside the float range).
__device__ __forceinline__ void bin_metric_d(const Program& P, int64_t i, double lp, double pv,
                                             double& term, double& fac) {
  const double n = P.bw[i], K = P.kbin;
  const bool lin = !P.root_log;
  if (P.metric == 0) {
    term = n == 0.0 ? 0.0 : -n * lp;
    fac = n == 0.0 ? 0.0 : (lin ? -n / pv : -n);
    return;
  }
  const double nu = K * pv;
  if (P.metric == 1) {
    term = n == 0.0 ? nu : nu - n * (lp + P.logk);
    fac = lin ? (n == 0.0 ? K : K - n / pv) : nu - n;
    return;
  }
  const double r = n - nu;
  term = r * r / P.bs2[i];
  fac = -2.0 * r * (lin ? K : nu) / P.bs2[i];
}

// ---- event stream ------------------------------------------------------------------------
// MODE 0: reduce -log P (and gradient) to result[0 .. nfree]; MODE 1: store log P_i;
// MODE 2: reduce the binned metric (the events are bin centres; Program.binned).
// Body of one (virtual) block vb of the vgrid blocks of an event launch.  Shared
// scratch: dyn (G: (kMaxStack + 1) nfree blockDim pairs/doubles), rec (leaf records in
// FP64), rf (the same as pairs), red[(blockDim / 32) (1 + kMaxFree1D)], *last.
// MX: 1 the program is an AddPdf of leaves (run_mixture only), 0 it is not (the stack
// machine only), -1 decided per launch from the program (the kernel holds both).
template <bool G, int MODE, int MX = -1>
__device__ __forceinline__ void events_1d_block(
    const Program& P, const WeidCoef& W, const Cols& cols, const int64_t n,
    const double* __restrict__ theta, const double* __restrict__ derived_g,
    double* __restrict__ partials, unsigned* __restrict__ counter, double* __restrict__ result,
    double* __restrict__ out_logp, const int32_t* __restrict__ perm, const int analytic_only,
    const int vb, const int vgrid, double* dyn, double* rec, F2* rf, double* red, int* last,
    F2* tay_smem) {
  const int bd = blockDim.x, tid = threadIdx.x;
  const int nf = P.nfree;
  constexpr int kRec = kMaxLeaf * kLeafRec + kMaxCoef;
  // leaf records: from the norm kernel, or (analytic leaves only) built here per block
  if (analytic_only) {
    if (tid < P.nleaf) make_leaf_record(P.leaf[tid], theta, 1.0, nullptr, rec + tid * kLeafRec);
    if (tid == 0) make_coefs(P, theta, rec + kMaxLeaf * kLeafRec);
  } else {
    for (int k = tid; k < kRec; k += bd) rec[k] = derived_g[k];
  }
  __syncthreads();
  for (int k = tid; k < kRec; k += bd) rf[k] = df_from(rec[k]);
  __syncthreads();
  F2* dynf = reinterpret_cast<F2*>(dyn);
  // per-thread gradient sums: after the interpreter's stack (kMaxStack levels of nf), or
  // for a mixture after its 4 x kMixMax component slots and the FP64 fallback's stack
  const int gbase = P.mix > 0 ? max(4 * kMixMax, kMaxStack * nf) : kMaxStack * nf;
  F2* gacc = dynf + (size_t)gbase * bd + tid;
  if (G)
    for (int k = 0; k < nf; ++k) gacc[k * bd] = F2{0.f, 0.f};
  F2 acc = {0.f, 0.f};

  // one event: log P_i into the sums (MODE 0, 2) or out_logp (MODE 1, through perm if
  // sorted)
  const bool mix = MX < 0 ? P.mix > 0 : MX == 1;
  const F2 kb = MODE == 2 ? df_split(P.kbin) : F2{0.f, 0.f};
  const F2 lk = MODE == 2 ? df_split(P.logk) : F2{0.f, 0.f};
  auto one_event = [&](int64_t i, const double* x, const Tay* tay) {
    const F2 s = mix ? run_mixture<G>(P, rec, rf, x, W, dynf + tid, bd, tay)
                     : run_program<ArF2, G>(P, rec, rf, x, W, dynf, nf, bd, tid, tay);
    // P in [2^-80, 2^125): every term that underflowed on the way (absolute error below
    // 2^-149 times a leaf constant) is negligible against P
    const bool ok = P.root_log ? (fabsf(s.hi) < 3.0e38f)
                               : (s.hi >= 8.271806125530277e-25f && s.hi < 4.2535295865117308e37f);
    if (ok) {
      const F2 lp = P.root_log ? s : df_log_tab(s, s_log_tab);
      if (MODE == 1) {
        out_logp[perm ? perm[i] : i] = df_to(lp);
      } else {
        F2 fac = {0.f, 0.f};
        if (MODE == 2) {
          F2 term;
          const F2 pv = P.root_log ? df_exp_tab(lp, s_exp_tab) : s;
          bin_metric_f2(P, i, lp, pv, kb, lk, term, fac);
          acc = df_add(acc, term);
        } else {
          acc = df_sub(acc, lp);
        }
        if (G) {
          const F2 sc = MODE == 2 ? fac : P.root_log ? F2{-1.f, 0.f} : df_neg(df_rcp(s));
          if (mix) {
            mixture_grad(P, rf, dynf + tid, sc, gacc, bd);
          } else {
            const F2* g0 = dynf + tid;
            for (int k = 0; k < nf; ++k)
              gacc[k * bd] = df_add(gacc[k * bd], df_mul(g0[k * bd], sc));
          }
        }
      }
    } else {
      // outside the float exponent range: this event again in FP64
      const double sd = run_program_fp64<G>(P, rec, x, W, dyn, nf, bd, tid);
      const double lp = P.root_log ? sd : df_log(sd);
      if (MODE == 1) {
        out_logp[perm ? perm[i] : i] = lp;
      } else {
        double fac = 0.0;
        if (MODE == 2) {
          double term;
          bin_metric_d(P, i, lp, P.root_log ? df_exp(sd) : sd, term, fac);
          acc = df_add(acc, df_from(term));
        } else {
          acc = df_sub(acc, df_from(lp));
        }
        if (G && (MODE != 2 || fac != 0.0)) {
          const double sc = MODE == 2 ? fac : P.root_log ? -1.0 : -1.0 / sd;
          const double* g0 = dyn + tid;
          for (int k = 0; k < nf; ++k)
            gacc[k * bd] = df_add(gacc[k * bd], df_from(g0[k * bd] * sc));
        }
      }
    }
  };

  const int64_t nthreads = (int64_t)vgrid * bd;
  const bool chunked = tay_smem && P.sorted && P.tay_slot >= 0 &&
                       n >= (int64_t)kChunk / 2 * nthreads;
  if (chunked) {
    // sorted events: thread g takes the contiguous share [n g / T, n (g + 1) / T), in
    // chunks of kChunk with one expansion of w per chunk
    Tay tay;
    tay.slot = P.tay_slot;
    tay.t = tay_smem + tid;
    tay.stride = bd;
    const int64_t g = (int64_t)vb * bd + tid;
    const int64_t lo = n * g / nthreads, hi = n * (g + 1) / nthreads;
    const double* xc = cols.c[P.tay_obs];
    const double* rv = rec + P.tay_slot * kLeafRec;
    const F2* fv = rf + P.tay_slot * kLeafRec;
    for (int64_t c0 = lo; c0 < hi; c0 += kChunk) {
      const int cnt = (int)(hi - c0 < kChunk ? hi - c0 : kChunk);
      const double xm = __ldg(xc + c0 + (cnt - 1) / 2);
      const float da = fabsf(__fmul_rn((float)(__ldg(xc + c0) - xm), fv[11].hi));
      const float db = fabsf(__fmul_rn((float)(__ldg(xc + c0 + cnt - 1) - xm), fv[11].hi));
      tay.ok = fmaxf(da, db) <= kTayLim;
      if (tay.ok) tay_build(tay, df_mul(df_split(xm - rv[10]), fv[11]), fv[12], W);
      for (int k = 0; k < cnt; ++k) {
        const int64_t i = c0 + k;
        double x[kMaxObs];
#pragma unroll
        for (int o = 0; o < kMaxObs; ++o)
          if (o < P.nobs) x[o] = __ldg(cols.c[o] + i);
        one_event(i, x, &tay);
      }
    }
  } else {
    const int64_t npairs = (n + 1) >> 1;
    for (int64_t pr = (int64_t)vb * bd + tid; pr < npairs; pr += nthreads) {
      double2 xv[kMaxObs];
      const bool full = 2 * pr + 1 < n;  // the last pair of an odd n holds one event
#pragma unroll
      for (int o = 0; o < kMaxObs; ++o)
        if (o < P.nobs) {
          if (full) {
            xv[o] = __ldcs(reinterpret_cast<const double2*>(cols.c[o]) + pr);
          } else {
            xv[o].x = __ldcs(cols.c[o] + 2 * pr);
            xv[o].y = 0.0;
          }
        }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int64_t i = 2 * pr + e;
        if (i >= n) break;
        double x[kMaxObs];
#pragma unroll
        for (int o = 0; o < kMaxObs; ++o) x[o] = e ? xv[o].y : xv[o].x;
        one_event(i, x, nullptr);
      }
    }
  }
  if (MODE == 1) return;

  const int m = 1 + (G ? nf : 0);
  const int stride_p = 1 + kMaxFree1D;
  block_sum_pairs([&](int k) -> F2 { return k == 0 ? acc : gacc[(k - 1) * bd]; }, m, red,
                  partials + (size_t)vb * stride_p);
  if (!arrive_last_of(counter, (unsigned)vgrid, last)) return;
  reduce_partials(partials, vgrid, stride_p, m, result);
  if (tid == 0) *counter = 0u;
}

template <bool G, int MODE, int MX = -1>
__global__ void __launch_bounds__(kThreads1D) k_events_1d(
    const Program* __restrict__ Pg, const __grid_constant__ WeidCoef W, const Cols cols,
    const int64_t n, const double* __restrict__ theta, const double* __restrict__ derived_g,
    double* __restrict__ partials, unsigned* __restrict__ counter, double* __restrict__ result,
    double* __restrict__ out_logp, const int32_t* __restrict__ perm, const int analytic_only) {
  extern __shared__ double dyn[];  // G: (kMaxStack + 1) * nfree * blockDim entries
  __shared__ Program P;
  __shared__ double rec[kMaxLeaf * kLeafRec + kMaxCoef];
  __shared__ F2 rf[kMaxLeaf * kLeafRec + kMaxCoef];
  __shared__ double red[(kThreads1D / 32) * (1 + kMaxFree1D)];
  __shared__ int last;
  __shared__ F2 tay_t[(kTayDeg + 1) * 2 * kThreads1D];
  load_df_tables();
  load_program(Pg, P);
  events_1d_block<G, MODE, MX>(P, W, cols, n, theta, derived_g, partials, counter, result,
                               out_logp, perm, analytic_only, blockIdx.x, gridDim.x, dyn, rec, rf,
                               red, &last, tay_t);
}

// ---- log-domain products of exponential and Gaussian leaves ----------------------------
// A program of the form LEAF, (LEAF, LMUL) x (K - 1) with exponential and Gaussian leaves
// (Listing 1's ExpPdf, Listing 2's ProdPdf of two of them) has
//   log P_i = sum_k l_k(x_i),  l = a x - log N (EXP),  l = -u^2/2 - log N,
//   u = (x - mu)/sigma (GAUSS),
// so each event needs a few pair operations and no stack.  Per event the kernel adds the
// data-dependent part of every l_k (a x, -u^2/2) and of its gradient (x; u/sigma,
// u^2/sigma) into register accumulators; the constants -log N and d log N/d theta of each
// leaf enter once per thread, times its event count.  Data enter through df_split_trunc.

// x as a pair on the integer and FP32 pipes only: hi = x truncated to 24 significant bits,
// lo = the 29-bit remainder m, formed as m_hi 2^23 + m_lo from two exact floats (the
// 2^23 + k bit trick; no conversion instruction) with one rounding (|hi + lo - x| <=
// 2^-47 |x|; |lo| < ulp(hi)).  |x| outside [2^-74, 2^127), zero included, takes the
// conversion path.
__device__ __forceinline__ F2 df_split_trunc(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
  if (e - 949u > 201u) return df_from_cold(d);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  // exponent field e - 896 (8 bits) and the top 23 mantissa bits, by one funnel shift
  const unsigned hb = ((unsigned)(b >> 29) - (896u << 23)) | sign;
  const unsigned scale = ((hb & 0x7f800000u) - (52u << 23)) | sign;  // +-2^(e - 1075)
  const unsigned m = (unsigned)b & 0x1fffffffu;
  const float ml = __fsub_rn(__uint_as_float(0x4b000000u | (m & 0x7fffffu)), 8388608.f);
  const float mh = __fsub_rn(__uint_as_float(0x4b000000u | (m >> 23)), 8388608.f);
  const float lo = __fmul_rn(__fmaf_rn(mh, 8388608.f, ml), __uint_as_float(scale));
  return {__uint_as_float(hb), lo};
}

// Running sum of pairs: the high parts by TwoSum, the low parts and rounding errors in a
// float, renormalised after every few terms (renorm) so that |lo| stays within a few
// ulp(hi): each term then adds at most ~2^-47 |sum| of rounding, n terms n 2^-47.
struct LazyAcc {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a, float e) {
    const F2 s = two_sum(hi, a);
    hi = s.hi;
    lo = __fadd_rn(lo, __fadd_rn(s.lo, e));
  }
  __device__ __forceinline__ void renorm() {
    const F2 s = two_sum(hi, lo);
    hi = s.hi;
    lo = s.lo;
  }
  __device__ __forceinline__ F2 get() const { return two_sum(hi, lo); }
};

// a * b as p + e (p = fl(a.hi b.hi), e = its error and the cross terms)
__device__ __forceinline__ void prod_pe(F2 a, F2 b, float& p, float& e) {
  p = __fmul_rn(a.hi, b.hi);
  e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
}

constexpr int kLogUnroll = 4;  // double2 loads in flight per thread and observable

// KM: leaves handled (1: a single leaf over one observable; kLogLeaf: the general form);
// KIND: the leaf kind when KM == 1 (L_EXP or L_GAUSS), 0: read from the program.
template <bool G, int KM, int KIND>
__global__ void __launch_bounds__(kThreads1D) k_events_logsum(
    const Program* __restrict__ Pg, const Cols cols, const int64_t n,
    const double* __restrict__ theta, double* __restrict__ partials,
    unsigned* __restrict__ counter, double* __restrict__ result) {
  __shared__ Program P;
  __shared__ double rec[kMaxLeaf * kLeafRec + kMaxCoef];
  __shared__ F2 rf[kMaxLeaf * kLeafRec];
  __shared__ double red[(kThreads1D / 32) * (1 + kMaxFree1D)];
  __shared__ int last;
  extern __shared__ F2 gsh[];  // G: nfree x blockDim pairs (the per-thread gradient sums)
  const int tid = threadIdx.x, bd = blockDim.x;
  load_program(Pg, P);
  // the leaf records and their float pairs, computed on the host with theta (leafrec.h)
  // and uploaded behind it
  {
    const double* hr = theta + P.rec_off;
    const F2* hp = reinterpret_cast<const F2*>(hr + kLogLeaf * kLeafRec);
    for (int k = tid; k < P.nleaf * kLeafRec; k += bd) {
      rec[k] = hr[k];
      rf[k] = hp[k];
    }
  }
  __syncthreads();

  const int K = KM == 1 ? 1 : P.nleaf;
  int kind[KM], ob[KM];
  F2 c0[KM], c1[KM];  // EXP: a; GAUSS: 1/sigma (c1 unused for EXP)
  double mu[KM];
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    const int s = k < K ? k : 0;  // leaf k: record slot k, instruction 2k - 1 (k > 0)
    kind[k] = KIND ? KIND : (k < K ? P.leaf[s].kind : 0);
    ob[k] = k < K ? P.leaf[s].obs : 0;
    c0[k] = rf[s * kLeafRec + 10];
    c1[k] = rf[s * kLeafRec + 11];
    mu[k] = rec[s * kLeafRec + 10];
  }
  LazyAcc v;
  LazyAcc g[KM][2];

  // one event: the data-dependent parts of log P and of its gradient
  auto event = [&](double x0, double x1) {
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      if (KM > 1 && k >= K) break;
      const double x = (KM > 1 && ob[k]) ? x1 : x0;
      float p, q;
      if (kind[k] == L_EXP) {
        const F2 X = df_split_trunc(x);
        prod_pe(c0[k], X, p, q);  // a x
        v.add(p, q);
        if (G) g[k][0].add(X.hi, X.lo);
      } else {  // L_GAUSS: u = (x - mu)/sigma from the exact difference
        const F2 U = df_mul(df_split(x - mu[k]), c1[k]);
        const F2 U2 = df_mul(U, U);
        v.add(-0.5f * U2.hi, -0.5f * U2.lo);  // -u^2/2
        if (G) {
          prod_pe(U, c1[k], p, q);  // u / sigma
          g[k][0].add(p, q);
          prod_pe(U2, c1[k], p, q);  // u^2 / sigma
          g[k][1].add(p, q);
        }
      }
    }
  };
  auto renorm = [&]() {
    v.renorm();
    if (G)
#pragma unroll
      for (int k = 0; k < KM; ++k) {
        g[k][0].renorm();
        g[k][1].renorm();
      }
  };

  const int64_t nfull = n >> 1;  // pairs holding two events
  const int64_t npairs = (n + 1) >> 1;
  const int64_t nthreads = (int64_t)gridDim.x * bd;
  const bool two = KM > 1 && P.nobs > 1;
  const double2* pa = reinterpret_cast<const double2*>(cols.c[0]);
  const double2* pb = reinterpret_cast<const double2*>(two ? cols.c[1] : cols.c[0]);
  int64_t p0 = (int64_t)blockIdx.x * bd + tid;
  // main loop: kLogUnroll full pairs per thread and iteration, loads first, no guards;
  // pointers advance by increments (no 64-bit multiplies in the loop)
  const int64_t step = kLogUnroll * nthreads;
  const int64_t span = p0 + (kLogUnroll - 1) * nthreads;
  const int iters = span < nfull ? (int)((nfull - 1 - span) / step + 1) : 0;
  int cnt = 2 * kLogUnroll * iters;
  {
    const double2* qa = pa + p0;
    const double2* qb = pb + p0;
    for (int it = 0; it < iters; ++it) {
      double2 xa[kLogUnroll], xb[kLogUnroll];
#pragma unroll
      for (int u = 0; u < kLogUnroll; ++u) {
        xa[u] = __ldcs(qa + u * nthreads);
        if (two) xb[u] = __ldcs(qb + u * nthreads);
        else xb[u] = xa[u];
      }
      qa += step;
      qb += step;
#pragma unroll
      for (int u = 0; u < kLogUnroll; ++u) {
        event(xa[u].x, xb[u].x);
        event(xa[u].y, xb[u].y);
      }
      renorm();
    }
  }
  p0 += (int64_t)iters * step;
  // the thread's remaining pairs (fewer than kLogUnroll), the last one possibly single
  for (int64_t pr = p0; pr < npairs; pr += nthreads) {
    if (pr < nfull) {
      const double2 a = __ldcs(pa + pr);
      const double2 b = two ? __ldcs(pb + pr) : a;
      event(a.x, b.x);
      event(a.y, b.y);
      cnt += 2;
    } else {
      const double a = __ldcs(cols.c[0] + 2 * pr);
      const double b = two ? __ldcs(cols.c[1] + 2 * pr) : a;
      event(a, b);
      cnt += 1;
    }
  }
  renorm();

  // constants once per thread: value + cnt sum_k (-log N_k); gradient - cnt dlogN/dtheta
  // (cnt < 2^24 per thread: exact as a float)
  const F2 fc = F2{(float)cnt, 0.f};
  F2 val = v.get();
#pragma unroll
  for (int k = 0; k < KM; ++k)
    if (k < K) val = df_sub(val, df_mul(fc, rf[k * kLeafRec + 1]));
  val = df_neg(val);  // -sum log P
  const int nf = P.nfree;
  if (G) {
    for (int j = 0; j < nf; ++j) gsh[j * bd + tid] = F2{0.f, 0.f};
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      if (k >= K) break;
      const Instr& I = P.ins[k == 0 ? 0 : 2 * k - 1];
      const int np = kind[k] == L_EXP ? 1 : 2;
#pragma unroll
      for (int j = 0; j < 2; ++j)
        if (j < np && I.gidx[j] >= 0) {
          F2& t = gsh[I.gidx[j] * bd + tid];
          t = df_sub(t, df_sub(g[k][j].get(), df_mul(fc, rf[k * kLeafRec + 2 + j])));
        }
    }
  }
  const int m = 1 + (G ? nf : 0);
  const int stride_p = 1 + kMaxFree1D;
  block_sum_pairs([&](int k) -> F2 { return k == 0 ? val : gsh[(k - 1) * bd + tid]; }, m, red,
                  partials + (size_t)blockIdx.x * stride_p);
  if (!arrive_last_of(counter, gridDim.x, &last)) return;
  reduce_partials(partials, gridDim.x, stride_p, m, result);
  if (tid == 0) *counter = 0u;
}

// the instantiation for a program (single exponential or Gaussian leaf, or the general form)
template <bool G>
static auto logsum_kernel(const Program& P) {
  if (P.nleaf == 1 && P.leaf[0].kind == L_EXP) return k_events_logsum<G, 1, L_EXP>;
  if (P.nleaf == 1 && P.leaf[0].kind == L_GAUSS) return k_events_logsum<G, 1, L_GAUSS>;
  return k_events_logsum<G, kLogLeaf, 0>;
}

// ---- ConvolutionPdf (Sec. 3): lattice tables ------------------------------------------
// k_conv_points: the model subtree at the J model points and the resolution subtree at the
// K offsets, in FP64 through the same interpreter (records from k_norm_1d), value and
// gradient over the conv's local parameters, stored as float pairs.  One thread per point;
// the first ceil(J / blockDim) blocks take model points, the rest resolution offsets.
__global__ void __launch_bounds__(kThreads1D) k_conv_points(const ConvDesc* __restrict__ cdp,
                                                            const __grid_constant__ WeidCoef W,
                                                            const double* __restrict__ derived_g) {
  extern __shared__ double dyn[];  // (kMaxStack + 1) nfree blockDim doubles
  __shared__ Program P;
  __shared__ double rec[kMaxLeaf * kLeafRec + kMaxCoef];
  const ConvDesc& cd = *cdp;
  const int bd = blockDim.x, tid = threadIdx.x;
  const int nbm = (cd.J + bd - 1) / bd;
  const bool model = (int)blockIdx.x < nbm;
  load_program(model ? cd.pm : cd.pr, P);
  for (int k = tid; k < kMaxLeaf * kLeafRec + kMaxCoef; k += bd) rec[k] = derived_g[k];
  __syncthreads();
  const int t = (model ? (int)blockIdx.x : (int)blockIdx.x - nbm) * bd + tid;
  const int npts = model ? cd.J : cd.K;
  if (t >= npts) return;
  double x[kMaxObs];
#pragma unroll
  for (int o = 0; o < kMaxObs; ++o) x[o] = 0.0;
  if (model) x[cd.mcol] = cd.lo + (t - cd.kmax) * cd.h;
  else x[kResidCol] = (cd.kmin + t) * cd.h;
  const int nf = P.nfree;
  double v = run_program<ArD, true>(P, rec, rec, x, W, dyn, nf, bd, tid);
  double sc = 1.0;
  if (P.root_log) {  // the subtree's value in the linear domain: e^s, gradient e^s ds
    v = df_exp(v);
    sc = v;
  }
  float2* out = model ? cd.mt : cd.rt;
  const float vh = __double2float_rn(v);
  out[t] = make_float2(vh, __double2float_rn(v - (double)vh));
  for (int l = 0; l < cd.nloc; ++l) {
    const double g = dyn[(size_t)cd.loc2free[l] * bd + tid] * sc;
    const float gh = __double2float_rn(g);
    out[(size_t)(1 + l) * npts + t] = make_float2(gh, __double2float_rn(g - (double)gh));
  }
}

// k_conv_sum: C_i = h sum_k r_k m_{i - kmin - k + kmax} and its gradient rows in float
// pairs, one warp per (lattice point, row) with the lanes splitting the offsets, the table
// in FP64; then the trapezoid normalisation N = h (C_0/2 + C_1 + ... + C_L/2) and dN by
// the last block in a fixed order, which writes the conv leaf's record: 1/N, log N,
// dlogN/dtheta_l, and the constants lo, 1/h, L and the table's address.
__global__ void __launch_bounds__(kThreads1D) k_conv_sum(const ConvDesc* __restrict__ cdp,
                                                         double* __restrict__ derived) {
  __shared__ double red[(kThreads1D / 32) * (1 + kMaxLocal)];
  __shared__ double sums[1 + kMaxLocal];
  __shared__ int last;
  const ConvDesc& cd = *cdp;
  const int tid = threadIdx.x, lane = tid & 31;
  const int K = cd.K, J = cd.J, L = cd.L, nq = 1 + cd.nloc;
  const int w = (int)((blockIdx.x * (unsigned)blockDim.x + tid) >> 5);
  if (w < (L + 1) * nq) {
    const int i = w / nq, q = w - i * nq;
    const int j0 = i - cd.kmin + cd.kmax;  // model index for offset k = 0 (then j0 - k)
    LazyAcc acc;
    // row q = 0: r with m; row q = l + 1: dr_l with m, then r with dm_l
    const float2* ra = cd.rt + (size_t)q * K;
    const float2* ma = cd.mt + j0;
    for (int k = lane; k < K; k += 32) {
      float p, e;
      const float2 x = ra[k], y = ma[-k];
      prod_pe(F2{x.x, x.y}, F2{y.x, y.y}, p, e);
      acc.add(p, e);
    }
    if (q > 0) {
      const float2* mb = cd.mt + (size_t)q * J + j0;
      for (int k = lane; k < K; k += 32) {
        float p, e;
        const float2 x = cd.rt[k], y = mb[-k];
        prod_pe(F2{x.x, x.y}, F2{y.x, y.y}, p, e);
        acc.add(p, e);
      }
    }
    F2 v = acc.get();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const F2 u = {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
      v = df_add(v, u);
    }
    if (lane == 0) {
      const double c = df_to(v) * cd.h;
      cd.ct[(size_t)q * (L + 1) + i] = c;
      cd.partials[w] = (i == 0 || i == L) ? 0.5 * c : c;  // [i][q]: trapezoid terms
    }
  }
  if (!arrive_last_of(cd.counter, gridDim.x, &last)) return;
  reduce_partials(cd.partials, L + 1, nq, nq, sums);
  __syncthreads();
  if (tid == 0) {
    double* r = derived + (size_t)cd.slot * kLeafRec;
    for (int k = 0; k < kLeafRec; ++k) r[k] = 0.0;
    const double N = sums[0] * cd.h;
    r[0] = 1.0 / N;
    r[1] = log(N);
    for (int l = 0; l < cd.nloc; ++l) r[2 + l] = sums[1 + l] * cd.h / N;
    r[10] = cd.lo;
    r[11] = 1.0 / cd.h;
    r[12] = L;
    r[13] = __longlong_as_double(reinterpret_cast<long long>(cd.ct));
    *cd.counter = 0u;
  }
}

cudaError_t launch_conv(const ConvDesc& host, const ConvDesc* dev, const WeidCoef& W, int nfree,
                        double* derived, cudaStream_t st) {
  // points: 32 threads per block, so that the FP64 work of the subtrees spreads over
  // many SMs (each SM issues 2 FP64 operations per clock)
  const int bp = 32;
  const int nb = (host.J + bp - 1) / bp + (host.K + bp - 1) / bp;
  const size_t dyn = (size_t)(kMaxStack + 1) * std::max(nfree, 1) * bp * sizeof(double);
  k_conv_points<<<nb, bp, dyn, st>>>(dev, W, derived);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t warps = (int64_t)(host.L + 1) * (1 + host.nloc);
  const int bd = kThreads1D;
  k_conv_sum<<<(int)((warps * 32 + bd - 1) / bd), bd, 0, st>>>(dev, derived);
  return cudaGetLastError();
}

// ---- grid-normalised nodes (MappedPdf, CompositePdf; Sec. 3) -------------------------
// k_gnorm: the node's body (sub-program) at the nbins midpoints of its observable in FP64
// with the gradient over the node's local parameters; per-block pair sums, the last block
// forms N = h sum and dN, and writes the node's record: 1/N, log N, dlogN/dtheta_l.
__global__ void __launch_bounds__(kThreads1D) k_gnorm(const GNormDesc* __restrict__ gdp,
                                                      const __grid_constant__ WeidCoef W,
                                                      double* __restrict__ derived) {
  extern __shared__ double dyn[];  // (kMaxStack + 1) nfree blockDim doubles
  __shared__ Program P;
  __shared__ double rec[kMaxLeaf * kLeafRec + kMaxCoef];
  __shared__ double red[(kThreads1D / 32) * (1 + kMaxLocal)];
  __shared__ double sums[1 + kMaxLocal];
  __shared__ int last;
  const GNormDesc& gd = *gdp;
  const int bd = blockDim.x, tid = threadIdx.x;
  load_program(gd.sub, P);
  for (int k = tid; k < kMaxLeaf * kLeafRec + kMaxCoef; k += bd) rec[k] = derived[k];
  __syncthreads();
  const int nf = P.nfree, nq = 1 + gd.nloc;
  const int b = blockIdx.x * bd + tid;
  F2 tr[1 + kMaxLocal];
  for (int q = 0; q < nq; ++q) tr[q] = F2{0.f, 0.f};
  if (b < gd.nbins) {
    double x[kMaxObs];
#pragma unroll
    for (int o = 0; o < kMaxObs; ++o) x[o] = 0.0;
    x[gd.mcol] = gd.lo + (b + 0.5) * gd.h;
    double v = run_program<ArD, true>(P, rec, rec, x, W, dyn, nf, bd, tid);
    double sc = 1.0;
    if (P.root_log) {
      v = df_exp(v);
      sc = v;
    }
    tr[0] = df_split(v);
    for (int l = 0; l < gd.nloc; ++l) tr[1 + l] = df_split(dyn[(size_t)gd.loc2free[l] * bd + tid] * sc);
  }
  const int stride = 1 + kMaxLocal;
  block_sum_pairs([&](int q) -> F2 { return tr[q]; }, nq, red,
                  gd.partials + (size_t)blockIdx.x * stride);
  if (!arrive_last_of(gd.counter, gridDim.x, &last)) return;
  reduce_partials(gd.partials, gridDim.x, stride, nq, sums);
  __syncthreads();
  if (tid == 0) {
    double* r = derived + (size_t)gd.slot * kLeafRec;
    for (int k = 0; k < kLeafRec; ++k) r[k] = 0.0;
    const double N = sums[0] * gd.h;
    r[0] = 1.0 / N;
    r[1] = log(N);
    for (int l = 0; l < gd.nloc; ++l) r[2 + l] = sums[1 + l] * gd.h / N;
    *gd.counter = 0u;
  }
}

cudaError_t launch_gnorm(const GNormDesc& host, const GNormDesc* dev, const WeidCoef& W,
                         int nfree, double* derived, cudaStream_t st) {
  const int bd = kThreads1D;
  const size_t dyn = (size_t)(kMaxStack + 1) * std::max(nfree, 1) * bd * sizeof(double);
  k_gnorm<<<(host.nbins + bd - 1) / bd, bd, dyn, st>>>(dev, W, derived);
  return cudaGetLastError();
}

// ---- batched tick: every waiting 1D fit in one persistent launch -----------------------
// Shared by the two tick kernels: find the item's fit and bring its program into shared
// memory when it changes (blocks walk the items in increasing order).
__device__ __forceinline__ const TickItem& tick_item(const TickItem* __restrict__ items, int nfits,
                                                     int it, int& cur, Program& Ps) {
  int f = 0;
  while (f + 1 < nfits && items[f + 1].item0 <= it) ++f;
  const TickItem& ti = items[f];
  if (f != cur) {
    __syncthreads();
    const int* src = reinterpret_cast<const int*>(&static_cast<const Fit1D*>(ti.fit)->P);
    int* dst = reinterpret_cast<int*>(&Ps);
    for (int k = threadIdx.x; k < (int)(sizeof(Program) / 4); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    cur = f;
  }
  return ti;
}

// normalisation grids of every batched fit (kThreads threads: one bin per thread)
__global__ void __launch_bounds__(kThreads, 1) k_tick_norm_1d(const TickItem* __restrict__ items,
                                                           int nfits, int total,
                                                           const __grid_constant__ WeidCoef W) {
  __shared__ Program Ps;
  __shared__ double red[32];
  __shared__ int last;
  __shared__ F2 sums[kMaxLeaf][4];
  __shared__ ShapeK shk;
  load_df_tables();  // visible after tick_item's first barrier
  int cur = -1;
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const TickItem& ti = tick_item(items, nfits, it, cur, Ps);
    const Fit1D* F = static_cast<const Fit1D*>(ti.fit);
    const int vb = it - ti.item0, ng = Ps.ngrid_blocks;
    if (vb >= ng) {  // the fit's table of w expansions (items beyond its grid blocks)
      const SBTabHdr& H = *reinterpret_cast<const SBTabHdr*>(ti.theta + Ps.rec_off);
      const int nt = (ti.nitems - ng) * blockDim.x;
      for (int j = (vb - ng) * blockDim.x + threadIdx.x; j < H.ntab; j += nt)
        sbtab_build(j, H, W, F->sbtab);
    } else {
      norm_1d_block(Ps, W, ti.theta, F->partials_norm, F->counter_norm, F->derived, vb, ng, red,
                    &last, sums, &shk);
    }
    __syncthreads();
  }
}

// event passes (NLL + gradient) of every batched fit (kThreads1D threads, as standalone)
// One instantiation per event-kernel mode, as the standalone launches (binned: MODE 2;
// unbinned: the AddPdf-of-leaves path MX = 1 or the stack machine MX = 0), so that a fit's
// blocks run the same code alone and batched and no instantiation carries every mode's
// registers.
template <int MODE, int MX>
__global__ void __launch_bounds__(kThreads1D) k_tick_events_1d(const TickItem* __restrict__ items,
                                                               int nfits, int total,
                                                               const __grid_constant__ WeidCoef W) {
  extern __shared__ double dyn[];
  __shared__ Program Ps;
  __shared__ double rec[kMaxLeaf * kLeafRec + kMaxCoef];
  __shared__ F2 rf[kMaxLeaf * kLeafRec + kMaxCoef];
  __shared__ double red[(kThreads1D / 32) * (1 + kMaxFree1D)];
  __shared__ int last;
  load_df_tables();  // visible after tick_item's first barrier
  int cur = -1;
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const TickItem& ti = tick_item(items, nfits, it, cur, Ps);
    const Fit1D* F = static_cast<const Fit1D*>(ti.fit);
    events_1d_block<true, MODE, MX>(Ps, W, F->cols, F->n, ti.theta, F->derived, F->partials,
                                    F->counter_ev, ti.result, nullptr, nullptr, F->analytic_only,
                                    it - ti.item0, ti.nitems, dyn, rec, rf, red, &last, nullptr);
    __syncthreads();
  }
}

cudaError_t launch_tick_1d(int kind, const TickItem* items, int nfits, int total,
                           const WeidCoef& W, size_t smem, int grid, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  switch (kind) {
    case kTick1DNorm: k_tick_norm_1d<<<grid, kThreads, 0, st>>>(items, nfits, total, W); break;
    case kTick1DStack:
      k_tick_events_1d<0, 0><<<grid, kThreads1D, smem, st>>>(items, nfits, total, W);
      break;
    case kTick1DMixture:
      k_tick_events_1d<0, 1><<<grid, kThreads1D, smem, st>>>(items, nfits, total, W);
      break;
    case kTick1DBinned:
      k_tick_events_1d<2, -1><<<grid, kThreads1D, smem, st>>>(items, nfits, total, W);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---- data check -------------------------------------------------------------------------------
struct Range {
  double lo[kMaxObs], hi[kMaxObs];
};
__global__ void k_check_range(const Cols cols, int nobs, int64_t n, const Range R, int* flag) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int o = 0; o < nobs; ++o) {
      const double v = cols.c[o][i];
      bad |= !(v >= R.lo[o] && v <= R.hi[o]);
    }
  // the flag lives in mapped pinned host memory: a plain store (every writer stores 1)
  if (__syncthreads_or(bad) && threadIdx.x == 0) *reinterpret_cast<volatile int*>(flag) = 1;
}

cudaError_t launch_check_range(const Cols& cols, int nobs, int64_t n, const double* lo,
                               const double* hi, int* flag, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  Range R{};
  for (int o = 0; o < nobs && o < kMaxObs; ++o) {
    R.lo[o] = lo[o];
    R.hi[o] = hi[o];
  }
  int64_t nb = (n + 255) / 256;
  if (nb > 152 * 8) nb = 152 * 8;
  k_check_range<<<(int)nb, 256, 0, st>>>(cols, nobs, n, R, flag);
  return cudaGetLastError();
}

// ---- host launchers ---------------------------------------------------------------------------
cudaError_t launch_norm_1d(const Program& P, const Program* prog, const WeidCoef& W,
                           const double* theta, double* partials, unsigned* counter,
                           double* derived, const SBTabHdr* tab_hdr, float4* tab,
                           int tab_blocks, cudaStream_t st) {
  const int nb = P.ngrid_blocks > 0 ? P.ngrid_blocks : 1;
  const int nt = tab ? tab_blocks : 0;
  k_norm_1d<<<nb + nt, kThreads, 0, st>>>(prog, W, theta, partials, counter, derived, nb,
                                           tab_hdr, tab);
  return cudaGetLastError();
}

size_t events_1d_smem(const Program& P, bool grad, int threads) {
  if (!grad) return 0;
  const int per = P.mix > 0 ? std::max(4 * kMixMax, kMaxStack * P.nfree) + P.nfree
                            : (kMaxStack + 1) * P.nfree;
  return (size_t)per * threads * sizeof(double);
}

cudaError_t launch_events_1d(const Program& P, const Program* prog, const WeidCoef& W,
                             const Cols& cols, int64_t n,
                             const double* theta, const double* derived, double* partials,
                             unsigned* counter, double* result, double* out_logp,
                             const int32_t* perm, bool grad, bool store, int analytic_only,
                             int nblocks, cudaStream_t st) {
  const int threads = kThreads1D;
  const size_t smem = events_1d_smem(P, grad, threads);
  if (P.binned && !store) {
    if (grad) {
      k_events_1d<true, 2><<<nblocks, threads, smem, st>>>(prog, W, cols, n, theta, derived,
                                                           partials, counter, result, out_logp,
                                                           nullptr, analytic_only);
    } else {
      k_events_1d<false, 2><<<nblocks, threads, 0, st>>>(prog, W, cols, n, theta, derived,
                                                         partials, counter, result, out_logp,
                                                         nullptr, analytic_only);
    }
  } else if (P.logsum && !store) {
    const size_t gs = grad ? sizeof(F2) * P.nfree * threads : 0;
    auto k = grad ? logsum_kernel<true>(P) : logsum_kernel<false>(P);
    k<<<nblocks, threads, gs, st>>>(prog, cols, n, theta, partials, counter, result);
  } else if (store) {
    k_events_1d<false, 1><<<nblocks, threads, 0, st>>>(prog, W, cols, n, theta, derived, partials,
                                                       counter, result, out_logp, perm,
                                                       analytic_only);
  } else {
    // AddPdf-of-leaves programs and the others in kernels of their own: each holds only its
    // path (fewer registers for the mixture, the headline workload)
    auto k = grad ? (P.mix ? k_events_1d<true, 0, 1> : k_events_1d<true, 0, 0>)
                  : (P.mix ? k_events_1d<false, 0, 1> : k_events_1d<false, 0, 0>);
    k<<<nblocks, threads, grad ? smem : 0, st>>>(prog, W, cols, n, theta, derived, partials,
                                                 counter, result, out_logp, nullptr,
                                                 analytic_only);
  }
  return cudaGetLastError();
}

// Opt the gradient kernels in to > 48 KB of dynamic shared memory on the current device.
// Called once per device when a context is created: never inside a stream capture.
cudaError_t prepare_kernels_1d() {
  cudaError_t e = upload_df_tables();
  auto attr = [&](const void* f) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  };
  attr((const void*)k_conv_points);
  attr((const void*)k_gnorm);
  attr((const void*)k_events_1d<true, 0, 0>);
  attr((const void*)k_events_1d<true, 0, 1>);
  attr((const void*)k_events_1d<true, 2>);
  attr((const void*)k_tick_events_1d<0, 0>);
  attr((const void*)k_tick_events_1d<0, 1>);
  attr((const void*)k_tick_events_1d<2, -1>);
  return e;
}

int events_logsum_blocks_per_sm(const Program& P) {
  int nb = 0;
  const size_t gs = sizeof(F2) * P.nfree * kThreads1D;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, logsum_kernel<true>(P), kThreads1D, gs);
  cudaGetLastError();
  return nb > 0 ? nb : 1;
}

int events_1d_blocks_per_sm(bool grad, size_t smem, bool mix) {
  int nb = 0;
  if (grad) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &nb, mix ? k_events_1d<true, 0, 1> : k_events_1d<true, 0, 0>, kThreads1D, smem);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &nb, mix ? k_events_1d<false, 0, 1> : k_events_1d<false, 0, 0>, kThreads1D, 0);
  }
  cudaGetLastError();
  return nb > 0 ? nb : 1;
}

}  // namespace gfi
