// k_dalitz.cu -- sm_103a kernels of the three-body Dalitz amplitude model (Sec. 4 of
// the paper: the D0 -> pi+ pi- pi0 analysis that drove GooFit's design).
//
//   A(s12, s13) = a_NR + sum_r c_r A_r,   A_r = F_L(q) S_L BW_r(s_ab),   P = |A|^2
//   NLL = -sum_i log P_i + n log N,        N = dA sum_{cells inside} |A(cell centre)|^2
//
// Kernels:
//   k_dalitz_mask      cell-centre-inside mask of the normalisation grid (set-up)
//   k_dalitz_ev_cache  per-event A_r of resonances whose shape (m0, Gamma0) is fixed
//   k_dalitz_grid_cols per-cell A_r of fixed-shape resonances (normalisation cache)
//   k_dalitz_gram      Gram matrix G_rs = dA sum conj(A_r) A_s from the cached columns:
//                      with every shape fixed, N = c^H G c costs O(K^2) per call
//   k_dalitz_stream    the event pass (METRIC_NLL / METRIC_STORE) or the direct norm
//                      pass over grid cells (METRIC_NORM) when some shape is free;
//                      FP64 or FP32 amplitudes (T), optional fused gradient (G)
#include <type_traits>

#include "devutil.cuh"
#include "gf_internal.h"
#include "launch.h"

namespace gfi {

enum Metric { METRIC_NLL = 0, METRIC_STORE = 1, METRIC_NORM = 2 };

template <typename T>
struct C2 {
  T r, i;
};

template <typename T>
__device__ __forceinline__ T rsq(T x);
template <>
__device__ __forceinline__ double rsq<double>(double x) { return rsqrt(x); }
template <>
__device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ DF rsq<DF>(DF x) { return df_rsqrt(x); }
template <typename T>
__device__ __forceinline__ T rcp(T x);
template <>
__device__ __forceinline__ double rcp<double>(double x) { return 1.0 / x; }
template <>
__device__ __forceinline__ float rcp<float>(float x) { return __frcp_rn(x); }
template <>
__device__ __forceinline__ DF rcp<DF>(DF x) { return df_rcp(x); }
template <typename T>
__device__ __forceinline__ T lg(T x);
template <>
__device__ __forceinline__ double lg<double>(double x) { return log(x); }
template <>
__device__ __forceinline__ float lg<float>(float x) { return logf(x); }
template <>
__device__ __forceinline__ DF lg<DF>(DF x) { return df_log_tab(x, s_log_tab); }
// an FP64 value in the arithmetic T (per block: conversion cost does not matter)
template <typename T>
__device__ __forceinline__ T conv(double v);
template <>
__device__ __forceinline__ double conv<double>(double v) { return v; }
template <>
__device__ __forceinline__ float conv<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ DF conv<DF>(double v) { return DF(df_from(v)); }
// an event coordinate (FP64 data) in T, per event: the pair split has no FP64 conversion
template <typename T>
__device__ __forceinline__ T ev_in(double v) { return conv<T>(v); }
template <>
__device__ __forceinline__ DF ev_in<DF>(double v) { return DF::from(v); }
template <typename T>
__device__ __forceinline__ double to_d(T v) { return (double)v; }
template <>
__device__ __forceinline__ double to_d<DF>(DF v) { return v.to_double(); }
template <typename T>
__device__ __forceinline__ T third() { return (T)(1.0 / 3.0); }
template <>
__device__ __forceinline__ DF third<DF>() { return DF(DFC(1.0 / 3.0)); }

// Per-call constants of one resonance, from theta (FP64 arithmetic, once per block).
struct ResK {
  double m0, m0sq, g0, cr, ci;
  double K;       // Gamma0 m0 B_L(z0) / q0^{2L+1}:  Gamma(m) = K q^{2L+1} / (m B_L(z))
  double sqrtB0;  // sqrt(B_L(z0)):                  F_L = sqrtB0 / sqrt(B_L(z))
  double hF;      // (1/2) d log B_L(z0)/dm0:        dF/dm0 = F hF
  double dlogK;   // d log K / dm0
  double invg0;
};

__device__ __forceinline__ double barrier(int L, double z) {
  return L == 0 ? 1.0 : (L == 1 ? 1.0 + z : fma(z, z + 3.0, 9.0));
}
__device__ __forceinline__ double barrier_dz(int L, double z) {
  return L == 0 ? 0.0 : (L == 1 ? 1.0 : fma(2.0, z, 3.0));
}

__device__ void res_constants(const DalitzPlan& D, const DalitzRes& R, const double* th, ResK& k) {
  const DalitzChannel& c = D.ch[R.channel];
  const int L = R.spin;
  const double m0 = th[R.p_m0], g0 = th[R.p_g0];
  const double u = m0 * m0;
  const double q02 = (u - c.thrA) * (u - c.thrB) / (4.0 * u);
  const double z0 = q02 * D.R2;
  const double B0 = barrier(L, z0);
  const double q0 = sqrt(q02);
  double q0p = q0;  // q0^{2L+1}
  for (int j = 0; j < L; ++j) q0p *= q02;
  k.m0 = m0;
  k.m0sq = u;
  k.g0 = g0;
  k.cr = th[R.p_re];
  k.ci = th[R.p_im];
  k.K = g0 * m0 * B0 / q0p;
  k.sqrtB0 = sqrt(B0);
  // d q0^2/dm0 = (m0^4 - thrA thrB)/(2 m0^3)
  const double dq02 = (u * u - c.thrA * c.thrB) / (2.0 * u * m0);
  const double dlogB0 = barrier_dz(L, z0) * D.R2 * dq02 / B0;
  k.hF = 0.5 * dlogB0;
  k.dlogK = 1.0 / m0 + dlogB0 - (2 * L + 1) * 0.5 * dq02 / q02;
  k.invg0 = 1.0 / g0;
}

// Per-event, per-channel kinematics (a, b = resonance pair; c = bachelor).
template <typename T>
struct ChanK {
  T sab, minv, q, qp1, qp2;  // s_ab, 1/m, q, q^3, q^5
  T rB1, iB1, rB2, iB2;      // 1/sqrt(B_1), 1/B_1, 1/sqrt(B_2), 1/B_2
  T S1, S2;
};

template <typename T>
__device__ __forceinline__ void chan_kin(const DalitzPlan& D, int ch, T s12, T s13, T s23,
                                         ChanK<T>& k) {
  const DalitzChannel& c = D.ch[ch];
  T sab, sbc, sac;
  if (ch == 0) { sab = s12; sbc = s23; sac = s13; }
  else if (ch == 1) { sab = s13; sbc = s23; sac = s12; }
  else { sab = s23; sbc = s13; sac = s12; }
  const T rs = rsq<T>(sab);
  const T inv_s = rs * rs;
  k.sab = sab;
  k.minv = rs;
  T q2 = (sab - (T)c.thrA) * (sab - (T)c.thrB) * inv_s * (T)0.25;
  q2 = q2 > (T)0 ? q2 : (T)0;
  const T rq = q2 > (T)0 ? rsq<T>(q2) : (T)0;
  k.q = q2 * rq;
  k.qp1 = k.q * q2;
  k.qp2 = k.qp1 * q2;
  const T z = q2 * (T)D.R2;
  const T B1 = (T)1 + z;
  const T B2 = z * (z + (T)3) + (T)9;
  k.rB1 = rsq<T>(B1);
  k.iB1 = k.rB1 * k.rB1;
  k.rB2 = rsq<T>(B2);
  k.iB2 = k.rB2 * k.rB2;
  k.S1 = sbc - sac + (T)c.k1 * inv_s;
  const T a2 = sab - (T)c.a2c + (T)c.a2k * inv_s;
  k.S2 = k.S1 * k.S1 - a2 * (T)4 * q2 * (T)(1.0 / 3.0);
}

// a b + c d and |z|^2 with every rounding explicit (float: one fma and one product)
template <typename T>
__device__ __forceinline__ T dot2(T a, T b, T c, T d) { return a * b + c * d; }
template <>
__device__ __forceinline__ float dot2<float>(float a, float b, float c, float d) {
  return __fmaf_rn(a, b, __fmul_rn(c, d));
}
template <typename T>
__device__ __forceinline__ T cabs2(const C2<T>& z) { return dot2<T>(z.r, z.r, z.i, z.i); }

// Per-block constants of the event pass in its arithmetic T (float or DF): channel
// constants of the plan and per-resonance constants from theta, converted once per block
// so that no event converts an FP64 value.
template <typename T>
struct DzC {
  T thrA[3], thrB[3], k1[3], a2c[3], a2k[3];
  T R2;
  T m0[kMaxRes], m0sq[kMaxRes], K[kMaxRes], sB[kMaxRes], cr[kMaxRes], ci[kMaxRes];
  T hF[kMaxRes], dDfac[kMaxRes], twom0[kMaxRes], invg0[kMaxRes];
};

// Threads 0..2 fill the channel constants, threads 0..nres-1 the resonance constants
// (rk already holds the FP64 per-call constants); a barrier must follow.
template <typename T>
__device__ __forceinline__ void fill_dzc(const DalitzPlan& D, const ResK* rk, DzC<T>& C) {
  const int t = threadIdx.x;
  if (t < 3) {
    const DalitzChannel& c = D.ch[t];
    C.thrA[t] = conv<T>(c.thrA);
    C.thrB[t] = conv<T>(c.thrB);
    C.k1[t] = conv<T>(c.k1);
    C.a2c[t] = conv<T>(c.a2c);
    C.a2k[t] = conv<T>(c.a2k);
  }
  if (t == 0) C.R2 = conv<T>(D.R2);
  if (t < D.nres) {
    const ResK& k = rk[t];
    C.m0[t] = conv<T>(k.m0);
    C.m0sq[t] = conv<T>(k.m0sq);
    C.K[t] = conv<T>(k.K);
    C.sB[t] = conv<T>(k.sqrtB0);
    C.cr[t] = conv<T>(k.cr);
    C.ci[t] = conv<T>(k.ci);
    C.hF[t] = conv<T>(k.hF);
    C.dDfac[t] = conv<T>(1.0 + k.m0 * k.dlogK);
    C.twom0[t] = conv<T>(2.0 * k.m0);
    C.invg0[t] = conv<T>(k.invg0);
  }
}

template <typename T>
__device__ __forceinline__ void chan_kin_c(const DzC<T>& C, int ch, T s12, T s13, T s23,
                                           ChanK<T>& k) {
  T sab, sbc, sac;
  if (ch == 0) { sab = s12; sbc = s23; sac = s13; }
  else if (ch == 1) { sab = s13; sbc = s23; sac = s12; }
  else { sab = s23; sbc = s13; sac = s12; }
  const T zero = T(0.f);
  const T rs = rsq<T>(sab);
  const T inv_s = rs * rs;
  k.sab = sab;
  k.minv = rs;
  T q2 = (sab - C.thrA[ch]) * (sab - C.thrB[ch]) * inv_s * T(0.25f);
  q2 = q2 > zero ? q2 : zero;
  const T rq = q2 > zero ? rsq<T>(q2) : zero;
  k.q = q2 * rq;
  k.qp1 = k.q * q2;
  k.qp2 = k.qp1 * q2;
  const T z = q2 * C.R2;
  const T B1 = T(1.f) + z;
  const T B2 = z * (z + T(3.f)) + T(9.f);
  k.rB1 = rsq<T>(B1);
  k.iB1 = k.rB1 * k.rB1;
  k.rB2 = rsq<T>(B2);
  k.iB2 = k.rB2 * k.rB2;
  k.S1 = sbc - sac + C.k1[ch] * inv_s;
  const T a2 = sab - C.a2c[ch] + C.a2k[ch] * inv_s;
  k.S2 = k.S1 * k.S1 - a2 * T(4.f) * q2 * third<T>();
}

// Breit-Wigner pieces of resonance r (event pass, arithmetic T = DF).
template <typename T>
__device__ __forceinline__ void res_amp_c(const DalitzRes& R, const DzC<T>& C, int r,
                                          const ChanK<T>& c, C2<T>& A, T& FS, C2<T>& BW,
                                          T& Gm) {
  const int L = R.spin;
  T qpow, iB, F, S;
  if (L == 0) { qpow = c.q; iB = T(1.f); F = T(1.f); S = T(1.f); }
  else if (L == 1) { qpow = c.qp1; iB = c.iB1; F = C.sB[r] * c.rB1; S = c.S1; }
  else { qpow = c.qp2; iB = c.iB2; F = C.sB[r] * c.rB2; S = c.S2; }
  Gm = C.K[r] * qpow * c.minv * iB;
  const T Dr = C.m0sq[r] - c.sab;
  const T mG = C.m0[r] * Gm;
  const T inv = rcp<T>(Dr * Dr + mG * mG);
  BW.r = Dr * inv;
  BW.i = mG * inv;
  FS = F * S;
  A.r = FS * BW.r;
  A.i = FS * BW.i;
}

// Breit-Wigner pieces of resonance r at an event: returns A_r, and (for the gradient)
// FS = F_L S_L, BW, Gamma(m).
template <typename T>
__device__ __forceinline__ void res_amp(const DalitzRes& R, const ResK& k, const ChanK<T>& c,
                                        C2<T>& A, T& FS, C2<T>& BW, T& Gm) {
  const int L = R.spin;
  T qpow, iB, F, S;
  if (L == 0) { qpow = c.q; iB = (T)1; F = (T)1; S = (T)1; }
  else if (L == 1) { qpow = c.qp1; iB = c.iB1; F = (T)k.sqrtB0 * c.rB1; S = c.S1; }
  else { qpow = c.qp2; iB = c.iB2; F = (T)k.sqrtB0 * c.rB2; S = c.S2; }
  Gm = (T)k.K * qpow * c.minv * iB;
  const T m0 = (T)k.m0;
  const T Dr = (T)k.m0sq - c.sab;
  const T mG = m0 * Gm;
  const T inv = rcp<T>(Dr * Dr + mG * mG);
  BW.r = Dr * inv;
  BW.i = mG * inv;
  FS = F * S;
  A.r = FS * BW.r;
  A.i = FS * BW.i;
}

// Cached columns: float2 per-event amplitudes of FP32 plans (wide = 0), double2 grid
// columns of every plan (wide = 1), per-event amplitudes of FP64 plans as two float
// pairs (re hi, re lo, im hi, im lo) in a float4 (wide = 2).
// FP32 plans: the theta-dependent constants enter as hi + lo float pairs.  A constant
// rounded once per call carries the same relative error into every event, so the FP32
// likelihood would jump by ~n x 6e-8 whenever the rounding of m0, K, c_r ... flips as
// theta moves; with the pairs it varies smoothly and only the per-event roundings
// (independent across events) remain.
struct ResKf {
  float m0h, m0l, m0sqh, m0sql, Kh, Kl, sBh, sBl, crh, crl, cih, cil;
};
__device__ __forceinline__ void split_const(double v, float& h, float& l) {
  h = (float)v;
  l = (float)(v - (double)h);
}
__device__ __forceinline__ void make_resf(const ResK& k, ResKf& f) {
  split_const(k.m0, f.m0h, f.m0l);
  split_const(k.m0sq, f.m0sqh, f.m0sql);
  split_const(k.K, f.Kh, f.Kl);
  split_const(k.sqrtB0, f.sBh, f.sBl);
  split_const(k.cr, f.crh, f.crl);
  split_const(k.ci, f.cih, f.cil);
}
__device__ __forceinline__ void res_amp_f(const DalitzRes& R, const ResKf& k, const ChanK<float>& c,
                                          C2<float>& A, float& FS, C2<float>& BW, float& Gm) {
  const int L = R.spin;
  float qpow, iB, rB, S;
  if (L == 0) { qpow = c.q; iB = 1.f; rB = 1.f; S = 1.f; }
  else if (L == 1) { qpow = c.qp1; iB = c.iB1; rB = c.rB1; S = c.S1; }
  else { qpow = c.qp2; iB = c.iB2; rB = c.rB2; S = c.S2; }
  const float g = qpow * c.minv * iB;
  Gm = fmaf(k.Kh, g, k.Kl * g);
  const float Dr = (k.m0sqh - c.sab) + k.m0sql;
  const float mG = fmaf(k.m0h, Gm, k.m0l * Gm);
  const float inv = __frcp_rn(fmaf(Dr, Dr, mG * mG));
  BW.r = Dr * inv;
  BW.i = mG * inv;
  const float F = (L == 0) ? 1.f : fmaf(k.sBh, rB, k.sBl * rB);
  FS = F * S;
  A.r = FS * BW.r;
  A.i = FS * BW.i;
}

template <typename T>
__device__ __forceinline__ C2<T> load_cached(const void* base, int64_t stride, int slot,
                                             int64_t i, int wide) {
  if constexpr (std::is_same<T, DF>::value) {
    if (wide == 2) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(base) + (size_t)slot * stride + i);
      return {DF(F2{v.x, v.y}), DF(F2{v.z, v.w})};
    }
    const double2 v = __ldg(reinterpret_cast<const double2*>(base) + (size_t)slot * stride + i);
    return {DF::from(v.x), DF::from(v.y)};
  } else {
    if (wide) {
      const double2 v = __ldg(reinterpret_cast<const double2*>(base) + (size_t)slot * stride + i);
      return {(T)v.x, (T)v.y};
    }
    const float2 v = __ldg(reinterpret_cast<const float2*>(base) + (size_t)slot * stride + i);
    return {(T)v.x, (T)v.y};
  }
}

// ---- set-up kernels --------------------------------------------------------------------------
// Inside test at a cell centre: |cos theta| <= 1 in the (12) rest frame, written as
// S_1^2 <= a2 a3 (4 k.q)^2 <= (4|k|^2)(4|q|^2) for channel (12), together with both
// invariant masses above threshold.
__device__ __forceinline__ bool inside_region(const DalitzPlan& D, double s12, double s13) {
  const double s23 = D.sum_m2 - s12 - s13;
  const DalitzChannel& c = D.ch[0];
  if (!(s12 > c.thrA) || !(s13 > D.ch[1].thrA) || !(s23 > D.ch[2].thrA)) return false;
  const double inv_s = 1.0 / s12;
  const double S1 = s23 - s13 + c.k1 * inv_s;
  const double a2 = s12 - c.a2c + c.a2k * inv_s;
  const double a3 = (s12 - c.thrA) * (s12 - c.thrB) * inv_s;
  return S1 * S1 <= a2 * a3;
}

__global__ void k_dalitz_mask(const DalitzPlan D, uint8_t* inside) {
  const int64_t ncell = (int64_t)D.nbx * D.nby;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ncell;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i / D.nby), iy = (int)(i % D.nby);
    const double s12 = D.x0 + (ix + 0.5) * D.hx, s13 = D.y0 + (iy + 0.5) * D.hy;
    inside[i] = inside_region(D, s12, s13) ? 1 : 0;
  }
}

__global__ void k_dalitz_check(const DalitzPlan D, const double* __restrict__ s12,
                               const double* __restrict__ s13, int64_t n, int* flag) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    bad |= !inside_region(D, s12[i], s13[i]);
  // the flag lives in mapped pinned host memory: a plain store (every writer stores 1)
  if (__syncthreads_or(bad) && threadIdx.x == 0) *reinterpret_cast<volatile int*>(flag) = 1;
}

__global__ void k_dalitz_fcols(const DalitzPlan D, const double* __restrict__ s12,
                               const double* __restrict__ s13, int64_t n, float* __restrict__ f) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = s12[i], b = s13[i];
    f[i] = (float)a;
    f[n + i] = (float)b;
    f[2 * n + i] = (float)(D.sum_m2 - a - b);
  }
}

// Per-event amplitudes of the event-cached resonances: FP64 values stored as float pairs
// (T = double, for the pair-arithmetic event pass) or FP32 (float2).
template <typename T>
__global__ void k_dalitz_ev_cache(const DalitzPlan D, const double* __restrict__ theta,
                                  const double* __restrict__ s12, const double* __restrict__ s13,
                                  int64_t n, void* __restrict__ cache) {
  __shared__ ResK rk[kMaxRes];
  if (threadIdx.x < D.nres) res_constants(D, D.res[threadIdx.x], theta, rk[threadIdx.x]);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = s12[i], b = s13[i];
    const double c = D.sum_m2 - a - b;
    ChanK<double> ck[3];
    for (int ch = 0; ch < 3; ++ch) chan_kin<double>(D, ch, a, b, c, ck[ch]);
    for (int r = 0; r < D.nres; ++r) {
      const DalitzRes& R = D.res[r];
      if (R.ev_cached < 0) continue;
      C2<double> A, BW;
      double FS, Gm;
      res_amp<double>(R, rk[r], ck[R.channel], A, FS, BW, Gm);
      if (sizeof(T) == 8) {
        const float rh = (float)A.r, ih = (float)A.i;
        reinterpret_cast<float4*>(cache)[(size_t)R.ev_cached * n + i] =
            make_float4(rh, (float)(A.r - (double)rh), ih, (float)(A.i - (double)ih));
      } else
        reinterpret_cast<float2*>(cache)[(size_t)R.ev_cached * n + i] =
            make_float2((float)A.r, (float)A.i);
    }
  }
}

// Per-cell amplitudes (FP64) of the listed resonances; zero outside the region.
__global__ void k_dalitz_grid_cols(const DalitzPlan D, const double* __restrict__ theta,
                                   const int* __restrict__ todo, int ntodo,
                                   double2* __restrict__ cols, const uint8_t* __restrict__ inside) {
  __shared__ ResK rk[kMaxRes];
  if (threadIdx.x < D.nres) res_constants(D, D.res[threadIdx.x], theta, rk[threadIdx.x]);
  __syncthreads();
  const int64_t ncell = (int64_t)D.nbx * D.nby;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ncell;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool in = inside[i] != 0;
    const int ix = (int)(i / D.nby), iy = (int)(i % D.nby);
    const double a = D.x0 + (ix + 0.5) * D.hx, b = D.y0 + (iy + 0.5) * D.hy;
    const double c = D.sum_m2 - a - b;
    for (int t = 0; t < ntodo; ++t) {
      const int r = todo[t];
      const DalitzRes& R = D.res[r];
      double2 v = make_double2(0.0, 0.0);
      if (in) {
        ChanK<double> ck;
        chan_kin<double>(D, R.channel, a, b, c, ck);
        C2<double> A, BW;
        double FS, Gm;
        res_amp<double>(R, rk[r], ck, A, FS, BW, Gm);
        v = make_double2(A.r, A.i);
      }
      cols[(size_t)(r + 1) * ncell + i] = v;
    }
  }
}

// Gram matrix from the columns: block (chunk, entry group of 8 upper-triangle entries).
// partials2[(chunk * ngroups + grp) * 16 + 2e + {0,1}] then the last block sums chunks.
constexpr int kGramGroup = 8;
__global__ void __launch_bounds__(kThreads) k_dalitz_gram(const DalitzPlan D,
                                                          const double2* __restrict__ cols,
                                                          const uint8_t* __restrict__ inside,
                                                          double* __restrict__ partials,
                                                          unsigned* __restrict__ counter,
                                                          double* __restrict__ gram, int nchunks) {
  __shared__ double red[32];
  __shared__ int last;
  const int K = D.nres + 1;
  const int nent = K * (K + 1) / 2;
  const int ngroups = (nent + kGramGroup - 1) / kGramGroup;
  const int chunk = blockIdx.x, grp = blockIdx.y;
  const int64_t ncell = (int64_t)D.nbx * D.nby;
  const int64_t per = (ncell + nchunks - 1) / nchunks;
  const int64_t beg = chunk * per, end = min(ncell, beg + per);
  int er[kGramGroup], es[kGramGroup];
  {
    int e = 0, idx = 0;
    for (int r = 0; r < K; ++r)
      for (int s = r; s < K; ++s, ++idx)
        if (idx >= grp * kGramGroup && idx < (grp + 1) * kGramGroup) {
          er[e] = r;
          es[e] = s;
          ++e;
        }
    for (; e < kGramGroup; ++e) er[e] = es[e] = -1;
  }
  double ar[kGramGroup], ai[kGramGroup];
#pragma unroll
  for (int e = 0; e < kGramGroup; ++e) ar[e] = ai[e] = 0.0;
  for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
    if (!inside[i]) continue;
#pragma unroll
    for (int e = 0; e < kGramGroup; ++e) {
      if (er[e] < 0) continue;
      const double2 x = er[e] == 0 ? make_double2(1.0, 0.0) : cols[(size_t)er[e] * ncell + i];
      const double2 y = es[e] == 0 ? make_double2(1.0, 0.0) : cols[(size_t)es[e] * ncell + i];
      // conj(x) y
      ar[e] = fma(x.x, y.x, fma(x.y, y.y, ar[e]));
      ai[e] = fma(x.x, y.y, fma(-x.y, y.x, ai[e]));
    }
  }
  for (int e = 0; e < kGramGroup; ++e) {
    const double r1 = block_sum(ar[e], red);
    const double r2 = block_sum(ai[e], red);
    if (threadIdx.x == 0) {
      partials[((size_t)chunk * ngroups + grp) * 2 * kGramGroup + 2 * e] = r1;
      partials[((size_t)chunk * ngroups + grp) * 2 * kGramGroup + 2 * e + 1] = r2;
    }
  }
  if (!arrive_last(counter, &last)) return;
  const double dA = D.hx * D.hy;
  for (int g = 0; g < ngroups; ++g)
    for (int e = 0; e < 2 * kGramGroup; ++e) {
      Neu a;
      for (int c = threadIdx.x; c < nchunks; c += blockDim.x)
        a.add(__ldcg(partials + ((size_t)c * ngroups + g) * 2 * kGramGroup + e));
      const double v = block_sum(a.get(), red);
      if (threadIdx.x == 0) {
        const int ent = g * kGramGroup + e / 2;
        if (ent < nent) {
          int idx = 0, rr = 0, ss = 0;
          for (int r = 0; r < K; ++r)
            for (int s = r; s < K; ++s, ++idx)
              if (idx == ent) { rr = r; ss = s; }
          const double val = v * dA;
          // G_rs and G_sr = conj(G_rs)
          const double im_part = (rr == ss) ? 0.0 : val;
          gram[2 * (rr * K + ss) + (e & 1)] = (e & 1) ? im_part : val;
          gram[2 * (ss * K + rr) + (e & 1)] = (e & 1) ? -im_part : val;
        }
      }
      __syncthreads();
    }
  if (threadIdx.x == 0) *counter = 0u;
}

// ---- the stream kernel ------------------------------------------------------------------------
// One pass over events (METRIC_NLL / METRIC_STORE) or over grid cells (METRIC_NORM).
// Per item: kinematics of the three channels, every resonance either loaded from its
// cache column or evaluated here, A = a_NR + sum c_r A_r, P = |A|^2; the metric is
// -log P (events) or P dA (cells); with G the partials d/dtheta as well.
// Shared memory: gacc[nfree][blockDim] per-thread gradient sums.
// Shared scratch of one block (static part).
template <typename T>
struct DzShared {
  ResK rk[kMaxRes];
  ResKf rkf[kMaxRes];
  DzC<T> C;
  double red[(kThreads / 32) * (1 + 4 * kMaxRes)];  // block_sum_pairs scratch
  double tot[1 + 4 * kMaxRes];
  double logN;
  double gv[2 * (kMaxRes + 1)];  // v_k = sum_s G_ks c_s (Gram normalisation), re/im
  int last;
  int need_ch[3];  // a channel's kinematics are needed by some resonance not cached
};

// c_k of the Gram form: c_0 = a_NR = 1, c_{r+1} = the resonance coefficients.
__device__ __forceinline__ void gram_coef(const ResK* rk, int k, double& cr, double& ci) {
  cr = k == 0 ? 1.0 : rk[k - 1].cr;
  ci = k == 0 ? 0.0 : rk[k - 1].ci;
}
// Threads k < K form v_k = sum_s G_ks c_s into gv (K = nres + 1); a barrier must follow.
__device__ __forceinline__ void gram_apply(const double* __restrict__ gram, const ResK* rk, int K,
                                           double* gv) {
  const int k = threadIdx.x;
  if (k < K) {
    double vr = 0.0, vi = 0.0;
    for (int s = 0; s < K; ++s) {
      double cr, ci;
      gram_coef(rk, s, cr, ci);
      const double gr = gram[2 * (k * K + s)], gi = gram[2 * (k * K + s) + 1];
      vr += gr * cr - gi * ci;
      vi += gr * ci + gi * cr;
    }
    gv[2 * k] = vr;
    gv[2 * k + 1] = vi;
  }
}

// FP64 plans with every resonance cached (fixed shapes): an event's cached amplitudes, the
// coefficients and the per-resonance gradient sums s conj(A) a_r (s = -2/|A|^2) held in
// registers (NR >= nres slots), A = 1 + sum c_r a_r accumulated as a lazily renormalised
// pair (each product's rounding error and each sum's carried in a float), the gradient
// sums renormalised every 16 events and added to the shared gradient slots once per
// thread.  Fewer operations and no shared-memory traffic per event than the general path.
__device__ __forceinline__ void lazy_prod(float& h, float& l, F2 a, F2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const F2 t = two_sum(h, p);
  h = t.hi;
  l = __fadd_rn(l, __fadd_rn(t.lo, e));
}
template <int NR, bool G>
__device__ __forceinline__ void cached_pairs_loop(const DalitzPlan& D, const DzC<DF>& C,
                                                  const void* __restrict__ cache,
                                                  int64_t stride, int64_t n, int vb, int vgrid,
                                                  Acc<DF>& acc, Acc<DF>* gacc, int bd) {
  const int nres = D.nres;
  F2 cr[NR], ci[NR], gr[NR], gi[NR];
  int slot[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    cr[r] = r < nres ? F2(C.cr[r]) : F2{0.f, 0.f};
    ci[r] = r < nres ? F2(C.ci[r]) : F2{0.f, 0.f};
    slot[r] = r < nres ? D.res[r].ev_cached : 0;
    gr[r] = gi[r] = F2{0.f, 0.f};
  }
  const float4* cq = reinterpret_cast<const float4*>(cache);
  int since = 0;
  for (int64_t i = (int64_t)vb * bd + threadIdx.x; i < n; i += (int64_t)vgrid * bd) {
    F2 ar[NR], ai[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r < nres) {
        const float4 v = __ldg(cq + (size_t)slot[r] * stride + i);
        ar[r] = F2{v.x, v.y};
        ai[r] = F2{v.z, v.w};
      } else {
        ar[r] = ai[r] = F2{0.f, 0.f};
      }
    }
    float hr = 1.f, lr = 0.f, hi = 0.f, li = 0.f;  // A = a_NR + sum c_r a_r
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r < nres) {
        lazy_prod(hr, lr, cr[r], ar[r]);
        lazy_prod(hr, lr, df_neg(ci[r]), ai[r]);
        lazy_prod(hi, li, cr[r], ai[r]);
        lazy_prod(hi, li, ci[r], ar[r]);
      }
    }
    const F2 Ar = fast_two_sum(hr, lr), Ai = fast_two_sum(hi, li);
    const F2 P = df_add(df_mul(Ar, Ar), df_mul(Ai, Ai));
    acc.add(df_neg(df_log_tab(P, s_log_tab)));
    if (G) {
      const F2 sc = df_mul_f(df_rcp(P), -2.f);
      const F2 Sr = df_mul(sc, Ar), Si = df_mul(sc, Ai);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (r < nres) {
          // s conj(A) a_r: real part to d/dRe c_r, Si ar - Sr ai to d/dIm c_r
          lazy_prod(gr[r].hi, gr[r].lo, Sr, ar[r]);
          lazy_prod(gr[r].hi, gr[r].lo, Si, ai[r]);
          lazy_prod(gi[r].hi, gi[r].lo, Si, ar[r]);
          lazy_prod(gi[r].hi, gi[r].lo, df_neg(Sr), ai[r]);
        }
      }
      if (++since == 16) {
        since = 0;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          gr[r] = fast_two_sum(gr[r].hi, gr[r].lo);
          gi[r] = fast_two_sum(gi[r].hi, gi[r].lo);
        }
      }
    }
  }
  if (G) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r < nres) {
        const DalitzRes& R = D.res[r];
        if (R.g_re >= 0) gacc[R.g_re * bd].add(DF(fast_two_sum(gr[r].hi, gr[r].lo)));
        if (R.g_im >= 0) gacc[R.g_im * bd].add(DF(fast_two_sum(gi[r].hi, gi[r].lo)));
      }
    }
  }
}

// Body of one (virtual) block vb of the vgrid blocks of a stream launch.  T = float (FP32
// plans: amplitudes in float with the hi/lo constants of ResKf) or DF (FP64 plans: every
// step in double-float pairs; only the event coordinates' differences enter in FP64).
// CO: every resonance comes from the event cache (fixed shapes): no kinematics, and the
// gradient pass reloads the amplitudes (L1 hits) instead of keeping them in registers.
template <typename T, bool G, int METRIC, bool CO = false>
__device__ __forceinline__ void dalitz_stream_block(
    const DalitzPlan& D, const double* __restrict__ theta, const double* __restrict__ s12d,
    const double* __restrict__ s13d, const float* __restrict__ sf, int64_t n,
    const void* __restrict__ cache, int64_t cache_stride, int cache_wide,
    const uint8_t* __restrict__ inside,
    double* __restrict__ partials, unsigned* __restrict__ counter, double* __restrict__ result,
    double* __restrict__ out_logp, double* __restrict__ norm_io, int norm_mode,
    const double* __restrict__ gram, const int vb, const int vgrid, double* dyn,
    DzShared<T>& sh) {
  constexpr bool kF = std::is_same<T, float>::value;
  ResK* rk = sh.rk;
  ResKf* rkf = sh.rkf;
  const DzC<T>& C = sh.C;
  double* red = sh.red;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int nf = D.nfree;
  const int nres = D.nres;
  if (tid < nres) {
    if constexpr (CO) {
      // every amplitude cached: only the coefficients enter (no running-width, barrier or
      // mass constants, whose FP64 square roots and divisions cost the prologue ~8 us)
      ResK& k = rk[tid];
      k.cr = theta[D.res[tid].p_re];
      k.ci = theta[D.res[tid].p_im];
      split_const(k.cr, rkf[tid].crh, rkf[tid].crl);
      split_const(k.ci, rkf[tid].cih, rkf[tid].cil);
    } else {
      res_constants(D, D.res[tid], theta, rk[tid]);
      make_resf(rk[tid], rkf[tid]);
    }
  }
  if (tid < 3) {
    int need = 0;
    for (int r = 0; r < nres; ++r) need |= (D.res[r].ev_cached < 0 && D.res[r].channel == tid);
    sh.need_ch[tid] = need;
  }
  Acc<T>* gacc = reinterpret_cast<Acc<T>*>(dyn) + tid;
  if (G)
    for (int k = 0; k < nf; ++k) gacc[k * bd] = Acc<T>();
  __syncthreads();
  if constexpr (CO) {
    if (tid < nres) {
      sh.C.cr[tid] = conv<T>(rk[tid].cr);
      sh.C.ci[tid] = conv<T>(rk[tid].ci);
    }
  } else {
    fill_dzc<T>(D, rk, sh.C);
  }
  if (METRIC == METRIC_STORE && norm_mode == DN_GRAM) gram_apply(gram, rk, nres + 1, sh.gv);
  __syncthreads();
  if (METRIC == METRIC_STORE && tid == 0) {
    // normalised log P: log |A|^2 - log N, N = c^H G c (Gram mode) or the direct pass
    double N = 0.0;
    if (norm_mode == DN_GRAM) {
      for (int k = 0; k <= nres; ++k) {
        double cr, ci;
        gram_coef(rk, k, cr, ci);
        N += cr * sh.gv[2 * k] + ci * sh.gv[2 * k + 1];
      }
    } else {
      N = norm_io[0];
    }
    sh.logN = log(N);
  }
  __syncthreads();
  const bool need0 = sh.need_ch[0] != 0, need1 = sh.need_ch[1] != 0, need2 = sh.need_ch[2] != 0;
  Acc<T> acc;
  // FP64 plans with every resonance cached: the register path above
  // (up to 8 resonances; larger models take the general path)
  constexpr bool kFastCached = CO && !kF && METRIC == METRIC_NLL;
  const bool fast = kFastCached && nres <= 8;
  if constexpr (kFastCached) {
    if (fast) cached_pairs_loop<8, G>(D, sh.C, cache, cache_stride, n, vb, vgrid, acc, gacc, bd);
  }
  const int64_t nitems = fast ? 0 : (METRIC == METRIC_NORM) ? (int64_t)D.nbx * D.nby : n;

  for (int64_t i = (int64_t)vb * bd + tid; i < nitems; i += (int64_t)vgrid * bd) {
    if constexpr (CO) {
      C2<T> At = {T(1.f), T(0.f)};  // a_NR
#pragma unroll
      for (int r = 0; r < kMaxRes; ++r) {
        if (r >= nres) break;
        const C2<T> Ar = load_cached<T>(cache, cache_stride, D.res[r].ev_cached, i, cache_wide);
        if constexpr (kF) {
          const ResKf& f = rkf[r];
          At.r = __fadd_rn(At.r, __fadd_rn(__fmaf_rn(f.crh, Ar.r, -__fmul_rn(f.cih, Ar.i)),
                                           __fmaf_rn(f.crl, Ar.r, -__fmul_rn(f.cil, Ar.i))));
          At.i = __fadd_rn(At.i, __fadd_rn(__fmaf_rn(f.crh, Ar.i, __fmul_rn(f.cih, Ar.r)),
                                           __fmaf_rn(f.crl, Ar.i, __fmul_rn(f.cil, Ar.r))));
        } else {
          At.r += C.cr[r] * Ar.r - C.ci[r] * Ar.i;
          At.i += C.cr[r] * Ar.i + C.ci[r] * Ar.r;
        }
      }
      // the serving tick runs this path in another kernel: float roundings are spelled
      // out (no contraction left to the compiler) so both give the same bits
      const T P = cabs2<T>(At);
      if (METRIC == METRIC_STORE) {
        out_logp[i] = to_d<T>(lg<T>(P)) - sh.logN;
        continue;
      }
      acc.add(-lg<T>(P));
      if (G) {
        const T sc = T(-2.f) * rcp<T>(P);
        const C2<T> As = {sc * At.r, sc * At.i};
#pragma unroll 1
        for (int r = 0; r < nres; ++r) {
          const DalitzRes& R = D.res[r];
          const C2<T> Ar = load_cached<T>(cache, cache_stride, R.ev_cached, i, cache_wide);
          // sc conj(A) A_r
          if (R.g_re >= 0) gacc[R.g_re * bd].add(dot2<T>(As.r, Ar.r, As.i, Ar.i));
          if (R.g_im >= 0) gacc[R.g_im * bd].add(dot2<T>(As.i, Ar.r, -As.r, Ar.i));
        }
      }
      continue;
    }
    T a, b, c;
    if (METRIC == METRIC_NORM) {
      if (!inside[i]) continue;
      const int ix = (int)(i / D.nby), iy = (int)(i % D.nby);
      const double da = D.x0 + (ix + 0.5) * D.hx, db = D.y0 + (iy + 0.5) * D.hy;
      a = ev_in<T>(da);
      b = ev_in<T>(db);
      c = ev_in<T>(D.sum_m2 - da - db);
    } else if constexpr (!kF) {
      const double da = __ldcs(s12d + i), db = __ldcs(s13d + i);
      a = ev_in<T>(da);
      b = ev_in<T>(db);
      c = ev_in<T>(D.sum_m2 - da - db);
    } else {
      a = __ldcs(sf + i);
      b = __ldcs(sf + n + i);
      c = __ldcs(sf + 2 * n + i);
    }
    ChanK<T> ck[3];
    if (need0) chan_kin_c<T>(C, 0, a, b, c, ck[0]);
    if (need1) chan_kin_c<T>(C, 1, a, b, c, ck[1]);
    if (need2) chan_kin_c<T>(C, 2, a, b, c, ck[2]);
    C2<T> Ar[kMaxRes], BW[kMaxRes];
    T FS[kMaxRes], Gm[kMaxRes];
    C2<T> At = {T(1.f), T(0.f)};  // a_NR
#pragma unroll
    for (int r = 0; r < kMaxRes; ++r) {
      if (r >= nres) break;
      const DalitzRes& R = D.res[r];
      if (R.ev_cached >= 0) {
        Ar[r] = load_cached<T>(cache, cache_stride, R.ev_cached, i, cache_wide);
      } else if constexpr (kF) {
        res_amp_f(R, rkf[r], ck[R.channel], Ar[r], FS[r], BW[r], Gm[r]);
      } else {
        res_amp_c<T>(R, C, r, ck[R.channel], Ar[r], FS[r], BW[r], Gm[r]);
      }
      if constexpr (kF) {
        const ResKf& f = rkf[r];
        const float ar = Ar[r].r, ai = Ar[r].i;
        At.r += fmaf(f.crh, ar, -f.cih * ai) + fmaf(f.crl, ar, -f.cil * ai);
        At.i += fmaf(f.crh, ai, f.cih * ar) + fmaf(f.crl, ai, f.cil * ar);
      } else {
        At.r += C.cr[r] * Ar[r].r - C.ci[r] * Ar[r].i;
        At.i += C.cr[r] * Ar[r].i + C.ci[r] * Ar[r].r;
      }
    }
    const T P = At.r * At.r + At.i * At.i;
    if (METRIC == METRIC_STORE) {
      out_logp[i] = to_d<T>(lg<T>(P)) - sh.logN;
      continue;
    }
    if (METRIC == METRIC_NLL) acc.add(-lg<T>(P));
    else acc.add(P);
    if (G) {
      // d P / d theta; events use d(-log P) = -(dP)/P, cells use dP
      const T sc = (METRIC == METRIC_NLL) ? T(-2.f) * rcp<T>(P) : T(2.f);
#pragma unroll
      for (int r = 0; r < kMaxRes; ++r) {
        if (r >= nres) break;
        const DalitzRes& R = D.res[r];
        // conj(A) A_r
        const T xr = At.r * Ar[r].r + At.i * Ar[r].i;
        const T xi = At.r * Ar[r].i - At.i * Ar[r].r;
        if (R.g_re >= 0) gacc[R.g_re * bd].add(sc * xr);
        if (R.g_im >= 0) gacc[R.g_im * bd].add(-(sc * xi));
        if (R.ev_cached < 0 && (R.g_m0 >= 0 || R.g_g0 >= 0)) {
          const T cr = C.cr[r], ci = C.ci[r];
          // BW^2
          const T b2r = BW[r].r * BW[r].r - BW[r].i * BW[r].i;
          const T b2i = T(2.f) * BW[r].r * BW[r].i;
          // conj(A) c_r
          const T yr = At.r * cr + At.i * ci;
          const T yi = At.r * ci - At.i * cr;
          if (R.g_m0 >= 0) {
            // dA_r/dm0 = FS (hF BW - BW^2 dD),  dD = 2 m0 - i Gamma (1 + m0 dlogK)
            const T dDr = C.twom0[r];
            const T dDi = -(Gm[r] * C.dDfac[r]);
            const T hF = C.hF[r];
            const T dr = FS[r] * (hF * BW[r].r - (b2r * dDr - b2i * dDi));
            const T di = FS[r] * (hF * BW[r].i - (b2r * dDi + b2i * dDr));
            gacc[R.g_m0 * bd].add(sc * (yr * dr - yi * di));
          }
          if (R.g_g0 >= 0) {
            // dA_r/dGamma0 = FS i m0 (Gamma/Gamma0) BW^2
            const T f = FS[r] * C.m0[r] * Gm[r] * C.invg0[r];
            const T dr = -(f * b2i), di = f * b2r;
            gacc[R.g_g0 * bd].add(sc * (yr * dr - yi * di));
          }
        }
      }
    }
  }
  if (METRIC == METRIC_STORE) return;

  const int m = 1 + (G ? nf : 0);
  // partials value-major: value k of block b at partials[k vgrid + b]
  block_sum_pairs([&](int k) { return k == 0 ? acc.pair() : gacc[(k - 1) * bd].pair(); }, m, red,
                  partials + vb, vgrid);
  // Gram normalisation: the first block done with its events forms N = c^H G c and dN
  // (serial FP64 work) and leaves them in norm_io before it arrives, off the last block's
  // path; the last block to arrive finds them there
  const bool gram_nll = METRIC == METRIC_NLL && norm_mode == DN_GRAM;
  if (gram_nll) {
    if (tid == 0) sh.last = atomicAdd(counter + 2, 1u) == 0u;
    __syncthreads();
    if (sh.last) {
      gram_apply(gram, rk, nres + 1, sh.gv);
      __syncthreads();
      if (tid == 0) {
        // N = c^H G c, c_0 = a_NR = 1;  v_k = sum_s G_ks c_s;  dN/dRe c_k = 2 Re v_k,
        // dN/dIm c_k = 2 Im v_k
        double N = 0.0;
        for (int k = 0; k < nf; ++k) norm_io[1 + k] = 0.0;
        for (int k = 0; k <= nres; ++k) {
          double cr, ci;
          gram_coef(rk, k, cr, ci);
          const double vr = sh.gv[2 * k], vi = sh.gv[2 * k + 1];
          N += cr * vr + ci * vi;  // Re(conj(c_k) v_k)
          if (k > 0 && G) {
            const DalitzRes& R = D.res[k - 1];
            if (R.g_re >= 0) norm_io[1 + R.g_re] += 2.0 * vr;
            if (R.g_im >= 0) norm_io[1 + R.g_im] += 2.0 * vi;
          }
        }
        norm_io[0] = N;
      }
    }
  }
  if (!arrive_last_of(counter, (unsigned)vgrid, &sh.last)) return;
  double* tot = sh.tot;
  reduce_partials(partials, vgrid, 1, m, tot, vgrid);
  __syncthreads();
  if (METRIC == METRIC_NORM) {
    const double dA = D.hx * D.hy;
    if (tid < m) result[tid] = tot[tid] * dA;
  } else {
    // combine with the normalisation (the Gram form's from the first block above, the
    // direct cell pass's otherwise): + n log N, + n dN/N, one value per thread
    const double N = __ldcg(norm_io);
    const double nn = (double)n;
    if (tid == 0) result[0] = tot[0] + nn * log(N);
    if (G)
      for (int k = tid; k < nf; k += bd) result[1 + k] = tot[1 + k] + nn * __ldcg(norm_io + 1 + k) / N;
  }
  if (tid == 0) {
    counter[0] = 0u;
    if (gram_nll) counter[2] = 0u;
  }
}

// Registers per variant (measured): pair (DF) event passes are held to 85 (3 blocks of
// 256 per SM) -- their dependent pair chains need the warps more than the registers --,
// FP32 ones to 128 (2 blocks); the pair cell pass keeps its registers (1 block).
// The cached-only FP64 event pass holds its amplitudes and gradient sums in registers
// (2 blocks).
template <typename T, bool G, int METRIC, bool CO>
constexpr int dz_min_blocks() {
  return std::is_same<T, DF>::value ? (METRIC == METRIC_NORM ? 1 : (CO && METRIC == METRIC_NLL ? 2 : 3))
                                    : 2;
}
template <typename T, bool G, int METRIC, bool CO>
__global__ void __launch_bounds__(kThreads, dz_min_blocks<T, G, METRIC, CO>()) k_dalitz_stream(
    const DalitzPlan D, const double* __restrict__ theta, const double* __restrict__ s12d,
    const double* __restrict__ s13d, const float* __restrict__ sf, int64_t n,
    const void* __restrict__ cache, int64_t cache_stride, int cache_wide,
    const uint8_t* __restrict__ inside,
    double* __restrict__ partials, unsigned* __restrict__ counter, double* __restrict__ result,
    double* __restrict__ out_logp, double* __restrict__ norm_io, int norm_mode,
    const double* __restrict__ gram) {
  extern __shared__ double dyn[];
  __shared__ DzShared<T> sh;
  load_df_tables();
  dalitz_stream_block<T, G, METRIC, CO>(D, theta, s12d, s13d, sf, n, cache, cache_stride,
                                        cache_wide, inside, partials, counter, result, out_logp,
                                        norm_io, norm_mode, gram, blockIdx.x, gridDim.x, dyn, sh);
}

// ---- batched tick: every waiting Dalitz fit (Gram normalisation) in one persistent launch
template <typename T>
__global__ void __launch_bounds__(kThreads) k_tick_dalitz(const TickItem* __restrict__ items,
                                                          int nfits, int total) {
  extern __shared__ double dyn[];
  __shared__ DalitzPlan Ds;
  __shared__ DzShared<T> sh;
  load_df_tables();
  int cur = -1;
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    int f = 0;
    while (f + 1 < nfits && items[f + 1].item0 <= it) ++f;
    const TickItem ti = items[f];
    const FitDz* F = static_cast<const FitDz*>(ti.fit);
    if (f != cur) {  // this fit's plan into shared memory
      __syncthreads();
      const int* src = reinterpret_cast<const int*>(&F->D);
      int* dst = reinterpret_cast<int*>(&Ds);
      for (int k = threadIdx.x; k < (int)(sizeof(DalitzPlan) / 4); k += blockDim.x) dst[k] = src[k];
      __syncthreads();
      cur = f;
    }
    dalitz_stream_block<T, true, METRIC_NLL, true>(Ds, ti.theta, F->s12, F->s13, F->sf, F->n,
                                             F->ev_cache, F->n, F->cache_wide, nullptr,
                                             F->partials, F->counter, ti.result, nullptr,
                                             F->norm_scratch, DN_GRAM, F->gram, it - ti.item0,
                                             ti.nitems, dyn, sh);
    __syncthreads();
  }
}

// ---- host launchers ---------------------------------------------------------------------------
static int grid_for(int64_t items, int threads, int cap) {
  int64_t b = (items + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

// Every launcher refuses (cudaErrorInvalidValue, nothing launched) a plan without a grid or
// a missing buffer, so a call on the wrong kind of context cannot reach the device.
cudaError_t launch_dalitz_mask(const DalitzPlan& D, uint8_t* inside, cudaStream_t st) {
  if (!inside || D.nbx <= 0 || D.nby <= 0) return cudaErrorInvalidValue;
  k_dalitz_mask<<<grid_for((int64_t)D.nbx * D.nby, 256, 4096), 256, 0, st>>>(D, inside);
  return cudaGetLastError();
}

cudaError_t launch_dalitz_check(const DalitzPlan& D, const double* s12, const double* s13,
                                int64_t n, int* flag, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_dalitz_check<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(D, s12, s13, n, flag);
  return cudaGetLastError();
}

cudaError_t launch_dalitz_fcols(const DalitzPlan& D, const double* s12, const double* s13,
                                int64_t n, float* fcols, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_dalitz_fcols<<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(D, s12, s13, n, fcols);
  return cudaGetLastError();
}

cudaError_t launch_dalitz_ev_cache(const DalitzPlan& D, bool mixed, const double* theta,
                                   const double* s12, const double* s13, int64_t n,
                                   void* ev_cache, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (!theta || !s12 || !s13 || !ev_cache) return cudaErrorInvalidValue;
  const int nb = grid_for(n, 256, 152 * 8);
  if (mixed) k_dalitz_ev_cache<float><<<nb, 256, 0, st>>>(D, theta, s12, s13, n, ev_cache);
  else k_dalitz_ev_cache<double><<<nb, 256, 0, st>>>(D, theta, s12, s13, n, ev_cache);
  return cudaGetLastError();
}

cudaError_t launch_dalitz_grid_cols(const DalitzPlan& D, const double* theta, const int* todo,
                                    int ntodo, void* grid_cols, const uint8_t* inside,
                                    cudaStream_t st) {
  if (ntodo <= 0) return cudaSuccess;
  if (!theta || !todo || !grid_cols || !inside || D.nbx <= 0 || D.nby <= 0)
    return cudaErrorInvalidValue;
  k_dalitz_grid_cols<<<grid_for((int64_t)D.nbx * D.nby, 256, 152 * 8), 256, 0, st>>>(
      D, theta, todo, ntodo, reinterpret_cast<double2*>(grid_cols), inside);
  return cudaGetLastError();
}

constexpr int kGramChunks = 304;
cudaError_t launch_dalitz_gram(const DalitzPlan& D, const DalitzBufs& B, cudaStream_t st) {
  if (!B.grid_cols || !B.inside || !B.partials2 || !B.counter2 || !B.gram || D.nbx <= 0 ||
      D.nby <= 0)
    return cudaErrorInvalidValue;
  const int K = D.nres + 1;
  const int ngroups = (K * (K + 1) / 2 + kGramGroup - 1) / kGramGroup;
  dim3 grid(kGramChunks, ngroups);
  k_dalitz_gram<<<grid, kThreads, 0, st>>>(D, reinterpret_cast<const double2*>(B.grid_cols),
                                          B.inside, B.partials2, B.counter2, B.gram, kGramChunks);
  return cudaGetLastError();
}

template <typename T, bool G, int M>
static cudaError_t launch_stream_t(const DalitzPlan& D, const double* theta, const DalitzBufs& B,
                                   const void* cache, int64_t cstride, int cwide, double* partials,
                                   unsigned* counter, double* result, int norm_mode, int nblocks,
                                   cudaStream_t st) {
  if (!theta || !partials || !counter || (M != METRIC_STORE && !result) ||
      (M == METRIC_STORE && !B.out_logp) || (B.n > 0 && (!B.s12 || !B.s13)))
    return cudaErrorInvalidValue;
  const size_t smem = G ? (size_t)D.nfree * kThreads * sizeof(Acc<T>) : 0;
  bool co = M != METRIC_NORM && D.nres > 0;
  for (int r = 0; r < D.nres; ++r) co = co && D.res[r].ev_cached >= 0;
  if (co && M != METRIC_NORM)
    k_dalitz_stream<T, G, M, true><<<nblocks, kThreads, smem, st>>>(
        D, theta, B.s12, B.s13, B.sf, B.n, cache, cstride, cwide, B.inside, partials, counter,
        result, B.out_logp, B.norm_out, norm_mode, B.gram);
  else
    k_dalitz_stream<T, G, M, false><<<nblocks, kThreads, smem, st>>>(
        D, theta, B.s12, B.s13, B.sf, B.n, cache, cstride, cwide, B.inside, partials, counter,
        result, B.out_logp, B.norm_out, norm_mode, B.gram);
  return cudaGetLastError();
}

cudaError_t launch_dalitz_norm_direct(const DalitzPlan& D, bool mixed, bool grad,
                                      const double* theta, const DalitzBufs& B, int nblocks,
                                      cudaStream_t st) {
  const int64_t ncell = (int64_t)D.nbx * D.nby;
  // cached grid columns: slot r -> column r + 1 (DalitzRes::grid_col); use ev_cached >= 0
  // as "column valid" by passing a plan whose ev_cached points at grid columns.
  DalitzPlan E = D;
  for (int r = 0; r < E.nres; ++r) E.res[r].ev_cached = D.res[r].ev_cached >= 0 ? r + 1 : -1;
  if (mixed) {
    if (grad)
      return launch_stream_t<float, true, METRIC_NORM>(E, theta, B, B.grid_cols, ncell, 1,
                                                         B.partials2, B.counter2, B.norm_out, 0,
                                                         nblocks, st);
    return launch_stream_t<float, false, METRIC_NORM>(E, theta, B, B.grid_cols, ncell, 1,
                                                        B.partials2, B.counter2, B.norm_out, 0,
                                                        nblocks, st);
  }
  if (grad)
    return launch_stream_t<DF, true, METRIC_NORM>(E, theta, B, B.grid_cols, ncell, 1,
                                                        B.partials2, B.counter2, B.norm_out, 0,
                                                        nblocks, st);
  return launch_stream_t<DF, false, METRIC_NORM>(E, theta, B, B.grid_cols, ncell, 1,
                                                       B.partials2, B.counter2, B.norm_out, 0,
                                                       nblocks, st);
}

cudaError_t launch_dalitz_events(const DalitzPlan& D, bool mixed, bool grad, bool store,
                                 int norm_mode, const double* theta, const DalitzBufs& B,
                                 int nblocks, cudaStream_t st) {
  const int64_t cs = B.n;
  if (store) {
    if (mixed)
      return launch_stream_t<float, false, METRIC_STORE>(D, theta, B, B.ev_cache, cs, mixed ? 0 : 2, B.partials,
                                                           B.counter, B.result, norm_mode,
                                                           nblocks, st);
    return launch_stream_t<DF, false, METRIC_STORE>(D, theta, B, B.ev_cache, cs, mixed ? 0 : 2, B.partials,
                                                          B.counter, B.result, norm_mode, nblocks,
                                                          st);
  }
  if (mixed) {
    if (grad)
      return launch_stream_t<float, true, METRIC_NLL>(D, theta, B, B.ev_cache, cs, mixed ? 0 : 2, B.partials,
                                                        B.counter, B.result, norm_mode, nblocks,
                                                        st);
    return launch_stream_t<float, false, METRIC_NLL>(D, theta, B, B.ev_cache, cs, mixed ? 0 : 2, B.partials,
                                                       B.counter, B.result, norm_mode, nblocks,
                                                       st);
  }
  if (grad)
    return launch_stream_t<DF, true, METRIC_NLL>(D, theta, B, B.ev_cache, cs, mixed ? 0 : 2, B.partials,
                                                       B.counter, B.result, norm_mode, nblocks,
                                                       st);
  return launch_stream_t<DF, false, METRIC_NLL>(D, theta, B, B.ev_cache, cs, mixed ? 0 : 2, B.partials,
                                                      B.counter, B.result, norm_mode, nblocks, st);
}

cudaError_t launch_tick_dalitz(bool mixed, const TickItem* items, int nfits, int total,
                               size_t smem, int grid, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  if (mixed) k_tick_dalitz<float><<<grid, kThreads, smem, st>>>(items, nfits, total);
  else k_tick_dalitz<DF><<<grid, kThreads, smem, st>>>(items, nfits, total);
  return cudaGetLastError();
}

// Opt the gradient kernels in to > 48 KB of dynamic shared memory on the current device.
// Called once per device when a context is created: never inside a stream capture.
static cudaError_t prepare_kernels_tddp();  // after the mixing kernels, below

cudaError_t prepare_kernels_dalitz() {
  cudaError_t e = upload_df_tables();
  const int lim = 160 * 1024;
  auto attr = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  };
  attr((const void*)k_dalitz_stream<float, true, METRIC_NLL, false>);
  attr((const void*)k_dalitz_stream<float, true, METRIC_NORM, false>);
  attr((const void*)k_dalitz_stream<DF, true, METRIC_NLL, false>);
  attr((const void*)k_dalitz_stream<DF, true, METRIC_NORM, false>);
  attr((const void*)k_dalitz_stream<float, true, METRIC_NLL, true>);
  attr((const void*)k_dalitz_stream<DF, true, METRIC_NLL, true>);
  attr((const void*)k_tick_dalitz<float>);
  attr((const void*)k_tick_dalitz<DF>);
  if (e == cudaSuccess) e = prepare_kernels_tddp();
  return e;
}

int dalitz_blocks_per_sm(bool mixed, bool grad, bool cached_only, int nfree) {
  int nb = 0;
  const size_t smem = grad ? (size_t)(nfree > 0 ? nfree : 1) * kThreads * 8 : 0;
  auto q = [&](const void* f, size_t sm) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kThreads, sm);
  };
  if (mixed) {
    if (cached_only) {
      if (grad) q((const void*)k_dalitz_stream<float, true, METRIC_NLL, true>, smem);
      else q((const void*)k_dalitz_stream<float, false, METRIC_NLL, true>, 0);
    } else {
      if (grad) q((const void*)k_dalitz_stream<float, true, METRIC_NLL, false>, smem);
      else q((const void*)k_dalitz_stream<float, false, METRIC_NLL, false>, 0);
    }
  } else {
    if (cached_only) {
      if (grad) q((const void*)k_dalitz_stream<DF, true, METRIC_NLL, true>, smem);
      else q((const void*)k_dalitz_stream<DF, false, METRIC_NLL, true>, 0);
    } else {
      if (grad) q((const void*)k_dalitz_stream<DF, true, METRIC_NLL, false>, smem);
      else q((const void*)k_dalitz_stream<DF, false, METRIC_NLL, false>, 0);
    }
  }
  cudaGetLastError();
  return nb > 0 ? nb : 1;
}

// ---- time-dependent Dalitz model (Sec. 4: the D0 -> pi+ pi- pi0 mixing fit) -------------
// Intensity I = 1/2 (|A|^2 + |B|^2) Tch + 1/2 (|A|^2 - |B|^2) Tc + Re(A* B) Tsh - Im(A* B) Ts,
// A = 1 + sum_r c_r a_r at (s12, s13), B the same sum at (s12, s23) (pi+ and pi- exchanged),
// Tch = (T(l1) + T(l2))/2, Tsh = (T(l1) - T(l2))/2, Tc + i Ts = T(l3), l1 = G(1 - y),
// l2 = G(1 + y), l3 = G(1 - i x), G = 1/tau, T(l) = e^{-l t} (t >= 0) convolved with a
// Gaussian of width s sigma_t; normalised over the Dalitz grid and all t, where the time
// integrals are 1/l.  FP64 throughout (the amplitudes come from a per-event cache, the
// resonance shapes being fixed).

// A complex FP64 value as two float pairs (re hi, re lo, im hi, im lo).
__device__ __forceinline__ float4 pair4(double re, double im) {
  const float a = __double2float_rn(re), c = __double2float_rn(im);
  return make_float4(a, __double2float_rn(re - (double)a), c, __double2float_rn(im - (double)c));
}

// Per-event amplitudes a_r, b_r: the resonance code of the Dalitz event pass in FP64,
// stored as float pairs (the event pass multiplies them in pair arithmetic).
__global__ void __launch_bounds__(kThreads) k_tddp_cache(const __grid_constant__ TddpPlan T,
                                                        const double* __restrict__ theta,
                                                        const double* __restrict__ s12,
                                                        const double* __restrict__ s13, int64_t n,
                                                        float4* __restrict__ cache) {
  const DalitzPlan& D = T.D;
  __shared__ ResK rk[kMaxRes];
  __shared__ DzC<double> C;
  if (threadIdx.x < D.nres) res_constants(D, D.res[threadIdx.x], theta, rk[threadIdx.x]);
  __syncthreads();
  fill_dzc<double>(D, rk, C);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = s12[i], y = s13[i], z = D.sum_m2 - x - y;
    for (int r = 0; r < D.nres; ++r) {
      const DalitzRes& R = D.res[r];
      ChanK<double> k;
      C2<double> A, BW;
      double FS, Gm;
      chan_kin_c<double>(C, R.channel, x, y, z, k);
      res_amp_c<double>(R, C, r, k, A, FS, BW, Gm);
      cache[(size_t)r * n + i] = pair4(A.r, A.i);
      chan_kin_c<double>(C, R.channel, x, z, y, k);  // (s12, s23): the CP-conjugate point
      res_amp_c<double>(R, C, r, k, A, FS, BW, Gm);
      cache[(size_t)(D.nres + r) * n + i] = pair4(A.r, A.i);
    }
  }
}

// Free resonance shapes: a_r, b_r and their derivatives in m0 and Gamma0, recomputed when
// a shape changes, in double-float pairs (the Dalitz pass's resonance code):
//   dA_r/dm0 = FS (hF BW - BW^2 dD), dD = 2 m0 - i Gamma (1 + m0 dlog K/dm0),
//   dA_r/dGamma0 = FS i m0 (Gamma/Gamma0) BW^2  (FS = F_L S_L).
__device__ __forceinline__ float4 pair4f(DF re, DF im) {
  return make_float4(re.hi, re.lo, im.hi, im.lo);
}
__device__ __forceinline__ void res_deriv_c(const DzC<DF>& C, int r, const DF& FS,
                                            const C2<DF>& BW, const DF& Gm, C2<DF>& dm,
                                            C2<DF>& dg) {
  const DF b2r = BW.r * BW.r - BW.i * BW.i, b2i = DF(2.f) * BW.r * BW.i;
  const DF dDr = C.twom0[r], dDi = -(Gm * C.dDfac[r]);
  dm.r = FS * (C.hF[r] * BW.r - (b2r * dDr - b2i * dDi));
  dm.i = FS * (C.hF[r] * BW.i - (b2r * dDi + b2i * dDr));
  const DF f = FS * C.m0[r] * Gm * C.invg0[r];
  dg.r = -(f * b2i);
  dg.i = f * b2r;
}

// cache[r n + i] = a_r, cache[(nres + r) n + i] = b_r; dcache[(4 r + j) n + i], j = 0..3:
// da_r/dm0, da_r/dGamma0, db_r/dm0, db_r/dGamma0 (float pairs).
__global__ void __launch_bounds__(kThreads) k_tddp_cache_free(const __grid_constant__ TddpPlan T,
                                                             const double* __restrict__ theta,
                                                             const double* __restrict__ s12,
                                                             const double* __restrict__ s13,
                                                             int64_t n, float4* __restrict__ cache,
                                                             float4* __restrict__ dcache) {
  const DalitzPlan& D = T.D;
  __shared__ ResK rk[kMaxRes];
  __shared__ DzC<DF> C;
  load_df_tables();
  if (threadIdx.x < D.nres) res_constants(D, D.res[threadIdx.x], theta, rk[threadIdx.x]);
  __syncthreads();
  fill_dzc<DF>(D, rk, C);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = s12[i], y = s13[i];
    const DF a = DF::from(x), b = DF::from(y), c = DF::from(D.sum_m2 - x - y);
    for (int r = 0; r < D.nres; ++r) {
      const DalitzRes& R = D.res[r];
      for (int side = 0; side < 2; ++side) {  // (s12, s13), then the CP-conjugate (s12, s23)
        ChanK<DF> k;
        C2<DF> A, BW, dm, dg;
        DF FS, Gm;
        if (side == 0) chan_kin_c<DF>(C, R.channel, a, b, c, k);
        else chan_kin_c<DF>(C, R.channel, a, c, b, k);
        res_amp_c<DF>(R, C, r, k, A, FS, BW, Gm);
        res_deriv_c(C, r, FS, BW, Gm, dm, dg);
        cache[(size_t)(side * D.nres + r) * n + i] = pair4f(A.r, A.i);
        dcache[(size_t)(4 * r + 2 * side) * n + i] = pair4f(dm.r, dm.i);
        dcache[(size_t)(4 * r + 2 * side + 1) * n + i] = pair4f(dg.r, dg.i);
      }
    }
  }
}

// Grid columns a_r, b_r at the cell centres inside the region (zero outside).
__global__ void __launch_bounds__(kThreads) k_tddp_gcols(const __grid_constant__ TddpPlan T,
                                                        const double* __restrict__ theta,
                                                        const uint8_t* __restrict__ inside,
                                                        double2* __restrict__ gcols) {
  const DalitzPlan& D = T.D;
  __shared__ ResK rk[kMaxRes];
  __shared__ DzC<double> C;
  if (threadIdx.x < D.nres) res_constants(D, D.res[threadIdx.x], theta, rk[threadIdx.x]);
  __syncthreads();
  fill_dzc<double>(D, rk, C);
  __syncthreads();
  const int64_t ncell = (int64_t)D.nbx * D.nby;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ncell;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i / D.nby), iy = (int)(i % D.nby);
    const double x = D.x0 + (ix + 0.5) * D.hx, y = D.y0 + (iy + 0.5) * D.hy;
    const double z = D.sum_m2 - x - y;
    for (int r = 0; r < D.nres; ++r) {
      double2 a = make_double2(0.0, 0.0), b = a;
      if (inside[i]) {
        const DalitzRes& R = D.res[r];
        ChanK<double> k;
        C2<double> A, BW;
        double FS, Gm;
        chan_kin_c<double>(C, R.channel, x, y, z, k);
        res_amp_c<double>(R, C, r, k, A, FS, BW, Gm);
        a = make_double2(A.r, A.i);
        chan_kin_c<double>(C, R.channel, x, z, y, k);
        res_amp_c<double>(R, C, r, k, A, FS, BW, Gm);
        b = make_double2(A.r, A.i);
      }
      gcols[(size_t)r * ncell + i] = a;
      gcols[(size_t)(D.nres + r) * ncell + i] = b;
    }
  }
}

// One block per entry (m, r, s) of the three matrices: dA sum_cells conj(u_r) v_s with
// (u, v) = (a, a), (b, b), (a, b) and index 0 the constant 1 (inside cells only), in a
// fixed order (per-thread FP64 sums, block_sum).
__global__ void __launch_bounds__(kThreads) k_tddp_gram(const __grid_constant__ TddpPlan T,
                                                       const uint8_t* __restrict__ inside,
                                                       const double2* __restrict__ gcols,
                                                       double2* __restrict__ gram) {
  const DalitzPlan& D = T.D;
  const int K1 = D.nres + 1;
  const int e = blockIdx.x, m = e / (K1 * K1), r = (e / K1) % K1, q = e % K1;
  const int64_t ncell = (int64_t)D.nbx * D.nby;
  const int ur = m == 1 ? 1 : 0, vs = m == 0 ? 0 : 1;  // 0: a columns, 1: b columns
  const double2* U = r > 0 ? gcols + (size_t)(ur * D.nres + r - 1) * ncell : nullptr;
  const double2* V = q > 0 ? gcols + (size_t)(vs * D.nres + q - 1) * ncell : nullptr;
  double sr = 0.0, si = 0.0;
  for (int64_t i = threadIdx.x; i < ncell; i += blockDim.x) {
    if (!inside[i]) continue;
    const double2 u = U ? U[i] : make_double2(1.0, 0.0);
    const double2 v = V ? V[i] : make_double2(1.0, 0.0);
    sr += u.x * v.x + u.y * v.y;  // conj(u) v
    si += u.x * v.y - u.y * v.x;
  }
  __shared__ double red[32];
  const double tr = block_sum(sr, red);
  __syncthreads();
  const double ti = block_sum(si, red);
  if (threadIdx.x == 0) gram[e] = make_double2(tr * D.hx * D.hy, ti * D.hx * D.hy);
}

// T(l; t, sigma) and dT/dl, dT/dsigma for complex l = (lr, li) (FP64; Faddeeva by
// Weideman's series for the complex rate, erfcx for real ones):
//   T = 1/2 e^{-t^2/(2 sigma^2)} w(i u), u = (l sigma^2 - t)/(sigma sqrt2), Re u >= 0,
//   T = e^{l^2 sigma^2/2 - l t} - 1/2 e^{-t^2/(2 sigma^2)} w(-i u), Re u < 0 (reflection);
//   dT/dl = (l sigma^2 - t) T - sigma/sqrt(2 pi) e^{-t^2/(2 sigma^2)},
//   dT/dsigma = l^2 sigma T - e^{-t^2/(2 sigma^2)} (l sigma^2 + t)/(sqrt(2 pi) sigma^2).
struct Cx {
  double r, i;
};
__device__ __forceinline__ Cx cmul(Cx a, Cx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ Cx cinv(Cx a) {
  const double d = 1.0 / (a.r * a.r + a.i * a.i);
  return {a.r * d, -a.i * d};
}
// g = e^{-t^2/(2 sigma^2)} and is = 1/sigma are the same for the three rates of an event
// and come in.
__device__ __forceinline__ void smeared_exp(Cx l, double t, double sig, double is, double g,
                                            const WeidCoef& W, Cx& T, Cx& dl, Cx& ds) {
  const double k = is * kInvSqrt2;
  const Cx u = {(l.r * sig * sig - t) * k, l.i * sig * sig * k};
  // One Faddeeva (or erfcx) evaluation at a selected argument, w(i u) or under reflection
  // w(-i u), i (sg u) = -sg Im u + i sg Re u: a warp holding events of both signs of Re u
  // (the usual case: Re u < 0 for t above l sigma^2) evaluates it once, not twice.
  const bool refl = u.r < 0.0;
  const double sg = refl ? -1.0 : 1.0;
  Cx w;
  if (l.i == 0.0) w = {erfcx_df(sg * u.r, W), 0.0};
  else faddeeva_df(-sg * u.i, sg * u.r, W, w.r, w.i);
  const double h = 0.5 * g * sg;
  T = {h * w.r, h * w.i};
  if (refl) {  // + e^{l^2 sigma^2/2 - l t}
    const double m = df_exp(0.5 * (l.r * l.r - l.i * l.i) * sig * sig - l.r * t);
    if (l.i == 0.0) {
      T.r += m;
    } else {
      double sn, cs;
      sincos(l.i * (l.r * sig * sig - t), &sn, &cs);
      T = {T.r + m * cs, T.i + m * sn};
    }
  }
  const double c = sig * kInvSqrt2Pi;  // sigma / sqrt(2 pi)
  const Cx a = {l.r * sig * sig - t, l.i * sig * sig};
  const Cx aT = cmul(a, T);
  dl = {aT.r - c * g, aT.i};
  const Cx l2 = cmul(l, l);
  const Cx l2T = cmul(l2, T);
  const double f = g * kInvSqrt2Pi * is * is;
  ds = {l2T.r * sig - f * (l.r * sig * sig + t), l2T.i * sig - f * (l.i * sig * sig)};
}

// The same for a real rate l, written out in real arithmetic.
__device__ __forceinline__ void smeared_exp_re(double l, double t, double sig, double is,
                                               double g, const WeidCoef& W, double& T,
                                               double& dl, double& ds) {
  const double a = l * sig * sig - t;
  const double u = a * is * kInvSqrt2;
  const bool refl = u < 0.0;
  T = (refl ? -0.5 : 0.5) * g * erfcx_df(fabs(u), W);
  if (refl) T += df_exp(0.5 * l * l * sig * sig - l * t);
  dl = a * T - sig * kInvSqrt2Pi * g;
  ds = l * l * sig * T - g * kInvSqrt2Pi * is * is * (l * sig * sig + t);
}

// Rates and their derivatives in (tau, x, y): l_j and dl_j/d(tau, x, y).
__device__ __forceinline__ void tddp_rates(double tau, double x, double y, Cx* l, Cx (*dl)[3]) {
  const double G = 1.0 / tau, G2 = G * G;
  l[0] = {G * (1 - y), 0.0};
  l[1] = {G * (1 + y), 0.0};
  l[2] = {G, -G * x};
  dl[0][0] = {-(1 - y) * G2, 0.0};
  dl[0][1] = {0.0, 0.0};
  dl[0][2] = {-G, 0.0};
  dl[1][0] = {-(1 + y) * G2, 0.0};
  dl[1][1] = {0.0, 0.0};
  dl[1][2] = {G, 0.0};
  dl[2][0] = {-G2, x * G2};
  dl[2][1] = {0.0, -G};
  dl[2][2] = {0.0, 0.0};
}

// The normalisation N(theta) and dN/dtheta_free, by the block, in three phases (each a
// short FP64 chain per thread; a serial chain on one thread costs the narrow FP64 pipe's
// full latency per operation):
//  1. thread (j, a), j < 4, a < K + 1: row a of v = M c for M = G_A, G_B, X (j = 0, 1, 2)
//     or of w = X^T conj(c) (j = 3) into vec[j (K + 1) + a];
//  2. thread 0: G_A = c^H G_A c, G_B, X = c^H X c, the time integrals 1/l_j and N;
//  3. thread e < 2 nres: the coefficient term e (Re, Im of c_{e/2}); threads 2 nres + q:
//     tau, x, y; into part[]; then thread k sums the terms of free parameter k in order
//     (a parameter may serve several coefficients).
// Nsh[0] = N, Nsh[1 + k] = dN/dtheta_k; scratch: vec[4 (kMaxRes + 1)], part[2 kMaxRes + 3],
// kd[8].  Called by every thread of the block; ends with a barrier.
__device__ void tddp_norm_block(const TddpPlan& T, const double* th, const double2* gram,
                                double* Nsh, Cx* vec, double* part, double* kd, bool grad) {
  const DalitzPlan& D = T.D;
  const int K1 = D.nres + 1, tid = threadIdx.x;
  auto coef = [&](int a) -> Cx {
    return a == 0 ? Cx{1.0, 0.0} : Cx{th[D.res[a - 1].p_re], th[D.res[a - 1].p_im]};
  };
  if (tid < 4 * K1) {
    const int j = tid / K1, a = tid % K1;
    // the row's entries first, all loads in flight (X_ba for w: conj(c_b) X_ba)
    double2 g[kMaxRes + 1];
#pragma unroll
    for (int b = 0; b < kMaxRes + 1; ++b)
      g[b] = b < K1 ? gram[j < 3 ? j * K1 * K1 + a * K1 + b : 2 * K1 * K1 + b * K1 + a]
                    : make_double2(0.0, 0.0);
    Cx v = {0.0, 0.0};
#pragma unroll
    for (int b = 0; b < kMaxRes + 1; ++b) {
      if (b >= K1) break;
      const Cx cb = coef(b);
      const Cx pr = j < 3 ? cmul({g[b].x, g[b].y}, cb) : cmul({cb.r, -cb.i}, {g[b].x, g[b].y});
      v = {v.r + pr.r, v.i + pr.i};
    }
    vec[tid] = v;
  }
  __syncthreads();
  if (tid == 0) {
    double GA = 0.0, GB = 0.0;
    Cx X = {0.0, 0.0};
    for (int k = 0; k < K1; ++k) {
      const Cx c = coef(k), cc = {c.r, -c.i};
      GA += cmul(cc, vec[k]).r;
      GB += cmul(cc, vec[K1 + k]).r;
      const Cx t = cmul(cc, vec[2 * K1 + k]);
      X = {X.r + t.r, X.i + t.i};
    }
    Cx l[3], dl[3][3];
    tddp_rates(th[T.p_tau], th[T.p_x], th[T.p_y], l, dl);
    const Cx i1 = cinv(l[0]), i2 = cinv(l[1]), i3 = cinv(l[2]);
    const double kk[4] = {0.5 * (i1.r + i2.r), i3.r, 0.5 * (i1.r - i2.r), i3.i};
    const double dI[4] = {0.5 * (GA + GB), 0.5 * (GA - GB), X.r, -X.i};
    Nsh[0] = dI[0] * kk[0] + dI[1] * kk[1] + dI[2] * kk[2] + dI[3] * kk[3];
    for (int k = 0; k < 4; ++k) {
      kd[k] = kk[k];
      kd[4 + k] = dI[k];
    }
  }
  __syncthreads();
  if (!grad) return;
  const int ne = 2 * D.nres;
  if (tid < ne) {
    // d/dRe c: 2 Re v, u + w; d/dIm c: 2 Im v, -i u + i w
    const int q = tid / 2 + 1, im = tid & 1;
    const Cx va = vec[q], vb = vec[K1 + q], ux = vec[2 * K1 + q], wx = vec[3 * K1 + q];
    const double dGA = 2.0 * (im ? va.i : va.r), dGB = 2.0 * (im ? vb.i : vb.r);
    const Cx dX = im ? Cx{ux.i - wx.i, -ux.r + wx.r} : Cx{ux.r + wx.r, ux.i + wx.i};
    part[tid] = 0.5 * (dGA + dGB) * kd[0] + 0.5 * (dGA - dGB) * kd[1] + dX.r * kd[2] -
                dX.i * kd[3];
  } else if (tid < ne + 3) {
    // d(1/l)/dq = -(1/l^2) dl/dq
    const int q = tid - ne;
    Cx l[3], dl[3][3];
    tddp_rates(th[T.p_tau], th[T.p_x], th[T.p_y], l, dl);
    Cx d[3];
    for (int j = 0; j < 3; ++j) {
      const Cx ij = cinv(l[j]);
      d[j] = cmul(cmul(ij, ij), dl[j][q]);
    }
    const double dk[4] = {-0.5 * (d[0].r + d[1].r), -d[2].r, -0.5 * (d[0].r - d[1].r), -d[2].i};
    part[tid] = kd[4] * dk[0] + kd[5] * dk[1] + kd[6] * dk[2] + kd[7] * dk[3];
  }
  __syncthreads();
  for (int k = tid; k < T.nfree; k += blockDim.x) {
    double v = 0.0;
    for (int e = 0; e < ne; ++e)
      if ((e & 1 ? D.res[e / 2].g_im : D.res[e / 2].g_re) == k) v += part[e];
    const int gp[3] = {T.g_tau, T.g_x, T.g_y};
    for (int q = 0; q < 3; ++q)
      if (gp[q] == k) v += part[ne + q];
    Nsh[1 + k] = v;
  }
  __syncthreads();
}

// Free resonance shapes: N(theta) and dN/dtheta_free by a direct pass over the cells
// inside the region (the Gram sums would change with every shape).  Per cell, in pairs,
// with the time integrals k = (Ich, Ic, Ish, Is) of the rates l_j (1/l_j):
//   I_c = p |A|^2 + q |B|^2 + Re(conj(A) B z),  p, q = (k0 +- k1)/2,  z = k2 + i k3,
//   dI/dRe c_r + i dI/dIm c_r = 2 (conj(a_r) E + conj(b_r) F),  E = p A + z B/2,
//   F = q B + conj(z) A/2,  dI/dshape_r = 2 Re(conj(E) c_r da_r + conj(F) c_r db_r),
// and for tau, x, y the sums of (|A|^2 + |B|^2)/2, (|A|^2 - |B|^2)/2, Re(conj(A) B),
// -Im(conj(A) B) times the derivatives of the k's.  The amplitudes are computed twice per
// cell (for A and B first, then with their derivatives for the gradient) rather than
// held.  Per-thread gradient sums in shared memory (nfree x blockDim pairs); the last
// block writes out[0] = N, out[1 + k] = dN/dtheta_k.
constexpr int kTddpNormStride = 5 + 4 * kMaxRes + 8;
__global__ void __launch_bounds__(kThreads) k_tddp_norm_direct(
    const __grid_constant__ TddpPlan T, const double* __restrict__ theta,
    const uint8_t* __restrict__ inside, double* __restrict__ partials,
    unsigned* __restrict__ counter, double* __restrict__ out) {
  const DalitzPlan& D = T.D;
  extern __shared__ F2 gsh[];  // nfree x blockDim
  __shared__ ResK rk[kMaxRes];
  __shared__ DzC<DF> C;
  __shared__ double red[(kThreads / 32) * kTddpNormStride];
  __shared__ double tot[kTddpNormStride];
  __shared__ int last;
  const int tid = threadIdx.x, bd = blockDim.x, nf = T.nfree, nres = D.nres;
  if (tid < nres) res_constants(D, D.res[tid], theta, rk[tid]);
  for (int k = 0; k < nf; ++k) gsh[k * bd + tid] = F2{0.f, 0.f};
  __syncthreads();
  fill_dzc<DF>(D, rk, C);
  __syncthreads();
  Cx l[3], dl[3][3];
  tddp_rates(theta[T.p_tau], theta[T.p_x], theta[T.p_y], l, dl);
  const Cx i1 = cinv(l[0]), i2 = cinv(l[1]), i3 = cinv(l[2]);
  const double k0 = 0.5 * (i1.r + i2.r), k1 = i3.r, k2 = 0.5 * (i1.r - i2.r), k3 = i3.i;
  const DF p = DF::from(0.5 * (k0 + k1)), q = DF::from(0.5 * (k0 - k1));
  const DF zr = DF::from(k2), zi = DF::from(k3), half = DF(0.5f), two = DF(2.f);
  DF sI = DF(0.f), sd[4] = {DF(0.f), DF(0.f), DF(0.f), DF(0.f)};
  const int64_t ncell = (int64_t)D.nbx * D.nby;
  for (int64_t i = (int64_t)blockIdx.x * bd + tid; i < ncell; i += (int64_t)gridDim.x * bd) {
    if (!inside[i]) continue;
    const int ix = (int)(i / D.nby), iy = (int)(i % D.nby);
    const double xd = D.x0 + (ix + 0.5) * D.hx, yd = D.y0 + (iy + 0.5) * D.hy;
    const DF a = DF::from(xd), b = DF::from(yd), c = DF::from(D.sum_m2 - xd - yd);
    ChanK<DF> ka[3], kb[3];
    for (int ch = 0; ch < 3; ++ch) {
      chan_kin_c<DF>(C, ch, a, b, c, ka[ch]);
      chan_kin_c<DF>(C, ch, a, c, b, kb[ch]);  // the CP-conjugate point (s12, s23)
    }
    C2<DF> A = {DF(1.f), DF(0.f)}, B = A;
    for (int r = 0; r < nres; ++r) {
      const DalitzRes& R = D.res[r];
      C2<DF> Ar, Br, BW;
      DF FS, Gm;
      res_amp_c<DF>(R, C, r, ka[R.channel], Ar, FS, BW, Gm);
      res_amp_c<DF>(R, C, r, kb[R.channel], Br, FS, BW, Gm);
      A.r += C.cr[r] * Ar.r - C.ci[r] * Ar.i;
      A.i += C.cr[r] * Ar.i + C.ci[r] * Ar.r;
      B.r += C.cr[r] * Br.r - C.ci[r] * Br.i;
      B.i += C.cr[r] * Br.i + C.ci[r] * Br.r;
    }
    const DF aa = A.r * A.r + A.i * A.i, bb = B.r * B.r + B.i * B.i;
    const DF xr = A.r * B.r + A.i * B.i, xi = A.r * B.i - A.i * B.r;  // conj(A) B
    sI += p * aa + q * bb + (xr * zr - xi * zi);
    sd[0] += half * (aa + bb);
    sd[1] += half * (aa - bb);
    sd[2] += xr;
    sd[3] += -xi;
    // E = p A + z B/2, F = q B + conj(z) A/2
    const C2<DF> E = {p * A.r + half * (zr * B.r - zi * B.i), p * A.i + half * (zr * B.i + zi * B.r)};
    const C2<DF> F = {q * B.r + half * (zr * A.r + zi * A.i), q * B.i + half * (zr * A.i - zi * A.r)};
    for (int r = 0; r < nres; ++r) {
      const DalitzRes& R = D.res[r];
      C2<DF> Ar, Br, BWa, BWb;
      DF FSa, Gma, FSb, Gmb;
      res_amp_c<DF>(R, C, r, ka[R.channel], Ar, FSa, BWa, Gma);
      res_amp_c<DF>(R, C, r, kb[R.channel], Br, FSb, BWb, Gmb);
      // conj(a) E + conj(b) F
      const DF ur = Ar.r * E.r + Ar.i * E.i + Br.r * F.r + Br.i * F.i;
      const DF ui = Ar.r * E.i - Ar.i * E.r + Br.r * F.i - Br.i * F.r;
      if (R.g_re >= 0) gsh[R.g_re * bd + tid] = df_add(gsh[R.g_re * bd + tid], two * ur);
      if (R.g_im >= 0) gsh[R.g_im * bd + tid] = df_add(gsh[R.g_im * bd + tid], two * ui);
      if (R.g_m0 >= 0 || R.g_g0 >= 0) {
        C2<DF> dma, dga, dmb, dgb;
        res_deriv_c(C, r, FSa, BWa, Gma, dma, dga);
        res_deriv_c(C, r, FSb, BWb, Gmb, dmb, dgb);
        // 2 Re(conj(E) c w_a + conj(F) c w_b) = 2 Re(c (conj(E) w_a + conj(F) w_b))
        auto term = [&](const C2<DF>& wa, const C2<DF>& wb) {
          const DF vr = E.r * wa.r + E.i * wa.i + F.r * wb.r + F.i * wb.i;
          const DF vi = E.r * wa.i - E.i * wa.r + F.r * wb.i - F.i * wb.r;
          return two * (C.cr[r] * vr - C.ci[r] * vi);
        };
        if (R.g_m0 >= 0) gsh[R.g_m0 * bd + tid] = df_add(gsh[R.g_m0 * bd + tid], term(dma, dmb));
        if (R.g_g0 >= 0) gsh[R.g_g0 * bd + tid] = df_add(gsh[R.g_g0 * bd + tid], term(dga, dgb));
      }
    }
  }
  const int m = 5 + nf;
  block_sum_pairs([&](int k) -> F2 {
                    return k == 0 ? F2(sI) : k < 5 ? F2(sd[k - 1]) : gsh[(k - 5) * bd + tid];
                  },
                  m, red, partials + blockIdx.x, gridDim.x);  // value-major
  if (!arrive_last_of(counter, gridDim.x, &last)) return;
  reduce_partials(partials, gridDim.x, 1, m, tot, gridDim.x);
  const double dA = D.hx * D.hy;
  if (tid == 0) out[0] = dA * tot[0];
  for (int k = tid; k < nf; k += bd) {
    double v = tot[5 + k];
    // tau, x, y: sum_k sd_k dk_k/dq, d(1/l)/dq = -(1/l^2) dl/dq
    const int gp[3] = {T.g_tau, T.g_x, T.g_y};
    for (int qq = 0; qq < 3; ++qq)
      if (gp[qq] == k) {
        Cx d[3];
        for (int j = 0; j < 3; ++j) {
          const Cx ij = cinv(l[j]);
          d[j] = cmul(cmul(ij, ij), dl[j][qq]);
        }
        v += tot[1] * (-0.5 * (d[0].r + d[1].r)) + tot[2] * (-d[2].r) +
             tot[3] * (-0.5 * (d[0].r - d[1].r)) + tot[4] * (-d[2].i);
      }
    out[1 + k] = dA * v;
  }
  if (tid == 0) *counter = 0u;
}

// The event pass: -log(I/N) summed (or stored per event) with the gradient; per-thread
// gradient sums in shared memory (nfree x blockDim pairs).  The amplitude sums A, B and
// the coefficient gradient (multiply-adds of cached amplitudes) run in double-float pairs
// on the FP32 pipe, the time dependence in FP64.  N enters the sums only through n log N
// and n dN/N, so the last block forms it after the events; a block that stores log P per
// event forms it first.
template <bool G, bool STORE>
__global__ void __launch_bounds__(kThreads, kTddpBlocksPerSm) k_tddp_events(
    const __grid_constant__ TddpPlan T, const __grid_constant__ WeidCoef W,
    const double* __restrict__ theta, const double* __restrict__ ct,
    const double* __restrict__ csig, int64_t n, const float4* __restrict__ cache,
    const float4* __restrict__ dcache, const double2* __restrict__ gram,
    const double* __restrict__ normd, double* __restrict__ nscratch, const double* __restrict__ c12,
    const double* __restrict__ c13, double* __restrict__ partials,
    unsigned* __restrict__ counter, double* __restrict__ result, double* __restrict__ out_logp) {
  const DalitzPlan& D = T.D;
  extern __shared__ F2 gsh[];  // G: nfree x blockDim
  __shared__ double th[4 * kMaxRes + 8];
  __shared__ double Nsh[1 + 4 * kMaxRes + 8];
  __shared__ double red[(kThreads / 32) * (1 + 4 * kMaxRes + 8)];
  __shared__ Cx vec[4 * (kMaxRes + 1)];
  __shared__ double part[2 * kMaxRes + 3], kd[8];
  __shared__ F2 cp[2 * kMaxRes];  // c_r as pairs (re, im)
  __shared__ int last;
  const int tid = threadIdx.x, bd = blockDim.x, nf = T.nfree;
  // theta_all holds at most 4 kMaxRes + 8 parameters for this model (checked at compile)
  for (int k = tid; k < 4 * kMaxRes + 8; k += bd) th[k] = theta[k];
  if (G)
    for (int k = 0; k < nf; ++k) gsh[k * bd + tid] = F2{0.f, 0.f};
  if (tid < 2 * D.nres)
    cp[tid] = df_split(theta[(tid & 1) ? D.res[tid >> 1].p_im : D.res[tid >> 1].p_re]);
  __syncthreads();
  double logN = 0.0;
  if (STORE) {
    if (normd) {
      logN = log(normd[0]);
    } else {
      tddp_norm_block(T, th, gram, Nsh, vec, part, kd, false);
      logN = log(Nsh[0]);
    }
  }
  const double tau = th[T.p_tau], mx = th[T.p_x], my = th[T.p_y], sc = th[T.p_s];
  Cx l[3], dl[3][3];
  tddp_rates(tau, mx, my, l, dl);
  const double gam = 1.0 / tau;
  Neu acc;
  // a contiguous share of floor(n / gridDim) or one more events per block (block b from
  // q b + floor(r b / gridDim), n = q gridDim + r): with every block resident
  // (kTddpBlocksPerSm per SM) each SM gets the same number of events to within 3
  const int64_t qb = n / gridDim.x, rb = n - qb * gridDim.x;
  const int64_t i_beg = qb * blockIdx.x + rb * blockIdx.x / gridDim.x;
  const int64_t i_end = qb * (blockIdx.x + 1) + rb * (blockIdx.x + 1) / gridDim.x;
  for (int64_t i = i_beg + tid; i < i_end; i += bd) {
    // A = 1 + sum_r c_r a_r, B = 1 + sum_r c_r b_r in pairs
    F2 Ar = {1.f, 0.f}, Ai = {0.f, 0.f}, Br = Ar, Bi = Ai;
    for (int r = 0; r < D.nres; ++r) {
      const float4 a = cache[(size_t)r * n + i], b = cache[(size_t)(D.nres + r) * n + i];
      const F2 cr = cp[2 * r], ci = cp[2 * r + 1];
      const F2 are = {a.x, a.y}, aim = {a.z, a.w}, bre = {b.x, b.y}, bim = {b.z, b.w};
      Ar = df_add(Ar, df_sub(df_mul(cr, are), df_mul(ci, aim)));
      Ai = df_add(Ai, df_add(df_mul(cr, aim), df_mul(ci, are)));
      Br = df_add(Br, df_sub(df_mul(cr, bre), df_mul(ci, bim)));
      Bi = df_add(Bi, df_add(df_mul(cr, bim), df_mul(ci, bre)));
    }
    const Cx A = {df_to(Ar), df_to(Ai)}, B = {df_to(Br), df_to(Bi)};
    const double t = ct[i], sigt = csig[i], sig = sc * sigt, is = 1.0 / sig;
    const double g = df_exp(-0.5 * t * t * is * is);
    // T_j, dT_j/dl_j, dT_j/dsigma for l_0,1 = G (1 -+ y) (real) and l_2 = G (1 - i x)
    double T0, T1, L0, L1, S0, S1;
    smeared_exp_re(l[0].r, t, sig, is, g, W, T0, L0, S0);
    smeared_exp_re(l[1].r, t, sig, is, g, W, T1, L1, S1);
    Cx T2, L2, S2;
    smeared_exp(l[2], t, sig, is, g, W, T2, L2, S2);
    const double kk[4] = {0.5 * (T0 + T1), T2.r, 0.5 * (T0 - T1), T2.i};
    const double aa = A.r * A.r + A.i * A.i, bb = B.r * B.r + B.i * B.i;
    const Cx X = cmul({A.r, -A.i}, B);
    const double dI[4] = {0.5 * (aa + bb), 0.5 * (aa - bb), X.r, -X.i};
    const double I = dI[0] * kk[0] + dI[1] * kk[1] + dI[2] * kk[2] + dI[3] * kk[3];
    // the sigma_t density: log D = 2 ll + log st - lam st - log Z, lam = e^ll,
    // ll = b0 + b1 u + b2 v, Z = e^{-lam slo} (1 + lam slo) - e^{-lam shi} (1 + lam shi)
    double logD = 0.0, dlam = 0.0, du = 0.0, dv = 0.0;
    if (T.dens) {
      du = c12[i] - T.sc;
      dv = c13[i] - T.sc;
      const double ll = th[T.p_b0] + th[T.p_b1] * du + th[T.p_b2] * dv;
      const double lam = df_exp(ll);
      const double el = df_exp(-lam * T.slo), eh = df_exp(-lam * T.shi);
      const double Z = el * (1.0 + lam * T.slo) - eh * (1.0 + lam * T.shi);
      logD = 2.0 * ll + df_log(sigt) - lam * sigt - df_log(Z);
      if (G) {
        const double dZ = lam * (T.shi * T.shi * eh - T.slo * T.slo * el);
        dlam = (2.0 / lam - sigt - dZ / Z) * lam;  // d log D / d ll
      }
    }
    if (STORE) {
      out_logp[i] = df_log(I) - logN + logD;
      continue;
    }
    acc.add(-df_log(I) - logD);
    if (G) {
      const double iI = -1.0 / I;
      // I = p |A|^2 + q |B|^2 + Re(z conj(A) B), p, q = (kk0 +- kk1)/2, z = kk2 + i kk3, so
      // dI/dconj(c_r) = conj(a_r) E + conj(b_r) F with E = p A + z B/2, F = q B + conj(z) A/2,
      // and dI/dRe c_r + i dI/dIm c_r = 2 dI/dconj(c_r).
      const double p = 0.5 * (kk[0] + kk[1]), q = 0.5 * (kk[0] - kk[1]);
      const Cx zB = cmul({kk[2], kk[3]}, B), zA = cmul({kk[2], -kk[3]}, A);
      const double f2 = 2.0 * iI;
      const F2 Er = df_split(f2 * (p * A.r + 0.5 * zB.r)), Ei = df_split(f2 * (p * A.i + 0.5 * zB.i));
      const F2 Fr = df_split(f2 * (q * B.r + 0.5 * zA.r)), Fi = df_split(f2 * (q * B.i + 0.5 * zA.i));
      for (int r = 0; r < D.nres; ++r) {
        const float4 a = cache[(size_t)r * n + i], b = cache[(size_t)(D.nres + r) * n + i];
        const F2 are = {a.x, a.y}, aim = {a.z, a.w}, bre = {b.x, b.y}, bim = {b.z, b.w};
        // conj(a) E + conj(b) F
        if (D.res[r].g_re >= 0) {
          F2& s = gsh[D.res[r].g_re * bd + tid];
          s = df_add(s, df_add(df_add(df_mul(are, Er), df_mul(aim, Ei)),
                               df_add(df_mul(bre, Fr), df_mul(bim, Fi))));
        }
        if (D.res[r].g_im >= 0) {
          F2& s = gsh[D.res[r].g_im * bd + tid];
          s = df_add(s, df_add(df_sub(df_mul(are, Ei), df_mul(aim, Er)),
                               df_sub(df_mul(bre, Fi), df_mul(bim, Fr))));
        }
      }
      // resonance shapes: Re(conj(E) c_r da_r + conj(F) c_r db_r) with the scaled E, F
      if (dcache)
        for (int r = 0; r < D.nres; ++r) {
          const DalitzRes& R = D.res[r];
          if (R.g_m0 < 0 && R.g_g0 < 0) continue;
          const F2 cr = cp[2 * r], ci = cp[2 * r + 1];
          for (int j = 0; j < 2; ++j) {
            const int gi = j ? R.g_g0 : R.g_m0;
            if (gi < 0) continue;
            const float4 da = dcache[(size_t)(4 * r + j) * n + i];
            const float4 db = dcache[(size_t)(4 * r + 2 + j) * n + i];
            const F2 dar = {da.x, da.y}, dai = {da.z, da.w}, dbr = {db.x, db.y}, dbi = {db.z, db.w};
            // w = c d (complex), then Re(conj(E) w_a) + Re(conj(F) w_b)
            const F2 war = df_sub(df_mul(cr, dar), df_mul(ci, dai));
            const F2 wai = df_add(df_mul(cr, dai), df_mul(ci, dar));
            const F2 wbr = df_sub(df_mul(cr, dbr), df_mul(ci, dbi));
            const F2 wbi = df_add(df_mul(cr, dbi), df_mul(ci, dbr));
            F2& sacc = gsh[gi * bd + tid];
            sacc = df_add(sacc, df_add(df_add(df_mul(Er, war), df_mul(Ei, wai)),
                                       df_add(df_mul(Fr, wbr), df_mul(Fi, wbi))));
          }
        }
      // the sigma_t density's parameters: d(-log D)/db = -(d log D/d ll) (1, u, v)
      if (T.dens) {
        if (T.g_b0 >= 0) gsh[T.g_b0 * bd + tid] = df_add(gsh[T.g_b0 * bd + tid], df_split(-dlam));
        if (T.g_b1 >= 0) gsh[T.g_b1 * bd + tid] = df_add(gsh[T.g_b1 * bd + tid], df_split(-dlam * du));
        if (T.g_b2 >= 0) gsh[T.g_b2 * bd + tid] = df_add(gsh[T.g_b2 * bd + tid], df_split(-dlam * dv));
      }
      // time parameters: dI = sum_k dI_k dkk_k with dkk from dT_j = dT_j/dl_j dl_j:
      // dl_j/dtau = -G l_j, dl_2/dx = -i G, dl_0,1/dy = -+ G; dT_j/ds = dT_j/dsigma sigma_t
      auto add_time = [&](int gi, double d0, double d1, Cx d2) {
        if (gi >= 0) {
          F2& s = gsh[gi * bd + tid];
          s = df_add(s, df_split((dI[0] * 0.5 * (d0 + d1) + dI[1] * d2.r +
                                  dI[2] * 0.5 * (d0 - d1) + dI[3] * d2.i) * iI));
        }
      };
      const Cx lL2 = cmul(L2, l[2]);
      add_time(T.g_tau, -gam * l[0].r * L0, -gam * l[1].r * L1, {-gam * lL2.r, -gam * lL2.i});
      add_time(T.g_x, 0.0, 0.0, {gam * L2.i, -gam * L2.r});
      add_time(T.g_y, -gam * L0, gam * L1, {0.0, 0.0});
      add_time(T.g_s, S0 * sigt, S1 * sigt, {S2.r * sigt, S2.i * sigt});
    }
  }
  if (STORE) return;
  const int m = 1 + (G ? nf : 0);
  block_sum_pairs([&](int k) -> F2 { return k == 0 ? df_split(acc.get()) : gsh[(k - 1) * bd + tid]; },
                  m, red, partials + blockIdx.x, gridDim.x);  // value-major
  if (!normd) {
    // fixed shapes: the first block done with its events forms N and dN from the Gram sums
    // (a serial FP64 stretch of ~13 us) and publishes them in nscratch before it arrives,
    // off the last block's path: the last block to arrive finds them there
    if (tid == 0) last = atomicAdd(counter + 2, 1u) == 0u;
    __syncthreads();
    if (last) {
      tddp_norm_block(T, th, gram, Nsh, vec, part, kd, G);
      for (int k = tid; k < 1 + nf; k += bd) nscratch[k] = Nsh[k];
    }
  }
  if (!arrive_last_of(counter, gridDim.x, &last)) return;
  reduce_partials(partials, gridDim.x, 1, m, result, gridDim.x);
  const double* nsrc = normd ? normd : nscratch;  // direct cell pass (free shapes) or above
  for (int k = tid; k < 1 + nf; k += bd) Nsh[k] = __ldcg(nsrc + k);
  __syncthreads();
  if (tid == 0) {
    result[0] += (double)n * log(Nsh[0]);
    counter[0] = 0u;
    counter[2] = 0u;
  }
  if (G)
    for (int k = tid; k < nf; k += bd) result[1 + k] += (double)n * Nsh[1 + k] / Nsh[0];
}

cudaError_t launch_tddp_cache(const TddpPlan& T, const double* theta, const double* s12,
                              const double* s13, int64_t n, float4* cache, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_tddp_cache<<<grid_for(n, kThreads, 152 * 8), kThreads, 0, st>>>(T, theta, s12, s13, n, cache);
  return cudaGetLastError();
}

cudaError_t launch_tddp_gram(const TddpPlan& T, const double* theta, const uint8_t* inside,
                             double2* gcols, double2* gram, cudaStream_t st) {
  const int64_t ncell = (int64_t)T.D.nbx * T.D.nby;
  k_tddp_gcols<<<grid_for(ncell, kThreads, 152 * 8), kThreads, 0, st>>>(T, theta, inside, gcols);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int K1 = T.D.nres + 1;
  k_tddp_gram<<<3 * K1 * K1, kThreads, 0, st>>>(T, inside, gcols, gram);
  return cudaGetLastError();
}

cudaError_t launch_tddp_events(const TddpPlan& T, bool grad, const double* theta,
                               const double* const* cols, int64_t n, const float4* cache,
                               const float4* dcache, const double2* gram, const double* normd,
                               double* nscratch, double* partials, unsigned* counter,
                               double* result, double* out_logp, int nblocks, const WeidCoef& W,
                               cudaStream_t st) {
  const size_t smem = grad ? sizeof(F2) * T.nfree * kThreads : 0;
  if (out_logp) {
    k_tddp_events<false, true><<<nblocks, kThreads, 0, st>>>(
        T, W, theta, cols[2], cols[3], n, cache, dcache, gram, normd, nscratch, cols[0], cols[1], partials,
        counter, result, out_logp);
  } else if (grad) {
    k_tddp_events<true, false><<<nblocks, kThreads, smem, st>>>(
        T, W, theta, cols[2], cols[3], n, cache, dcache, gram, normd, nscratch, cols[0], cols[1], partials,
        counter, result, nullptr);
  } else {
    k_tddp_events<false, false><<<nblocks, kThreads, 0, st>>>(
        T, W, theta, cols[2], cols[3], n, cache, dcache, gram, normd, nscratch, cols[0], cols[1], partials,
        counter, result, nullptr);
  }
  return cudaGetLastError();
}

cudaError_t launch_tddp_cache_free(const TddpPlan& T, const double* theta, const double* s12,
                                   const double* s13, int64_t n, float4* cache, float4* dcache,
                                   cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_tddp_cache_free<<<grid_for(n, kThreads, 152 * 8), kThreads, 0, st>>>(T, theta, s12, s13, n,
                                                                         cache, dcache);
  return cudaGetLastError();
}

cudaError_t launch_tddp_norm_direct(const TddpPlan& T, const double* theta,
                                    const uint8_t* inside, double* partials, unsigned* counter,
                                    double* out, int nblocks, cudaStream_t st) {
  const size_t smem = sizeof(F2) * (size_t)(T.nfree > 0 ? T.nfree : 1) * kThreads;
  k_tddp_norm_direct<<<nblocks, kThreads, smem, st>>>(T, theta, inside, partials, counter, out);
  return cudaGetLastError();
}

// The mixing kernels whose gradient sums in shared memory may exceed 48 KB (nfree x 256
// pairs, up to 56 parameters).
static cudaError_t prepare_kernels_tddp() {
  const int lim = 120 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_tddp_events<true, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tddp_norm_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  return e;
}

}  // namespace gfi
