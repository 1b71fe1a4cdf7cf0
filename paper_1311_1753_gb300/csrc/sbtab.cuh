// sbtab.cuh -- Taylor expansions of the Faddeeva function w(z) (Sec. 4: the Voigtian
// line shape) and the table of them along the line Im z = y of one evaluation.
//
// Around z0 = x0 + i y, w(z0 + d) = sum_k t_k d^k with t_k = w^(k)(z0)/k!; the differential
// equation w' = -2 z w + 2i/sqrt(pi) gives t_1 = -2 z0 t_0 + 2i/sqrt(pi) and
// t_{k+1} = -2 (z0 t_k + t_{k-1})/(k + 1).  For real d the real and imaginary parts of the
// sum separate.  The signal + background kernel either expands w once per chunk of sorted
// events, or (the table, SBTabHdr) looks each event's expansion up by its cell of Re z:
// both keep |d| within the limits validated against a 30-digit w (k_sigbkg.cu).
#pragma once
#include "devutil.cuh"

namespace gfi {

// t_0 .. t_DEG in pairs (the recurrence cancels at large |z0|).
template <int DEG>
__device__ __forceinline__ void tay_coefs(F2 zr, F2 y, const WeidCoef& W, F2* tr, F2* ti) {
  faddeeva_f2(zr, y, W, tr[0], ti[0]);
  F2 ar = df_sub(df_mul(zr, tr[0]), df_mul(y, ti[0]));
  F2 ai = df_add(df_mul(zr, ti[0]), df_mul(y, tr[0]));
  tr[1] = df_mul_f(ar, -2.f);
  ti[1] = df_add(df_mul_f(ai, -2.f), DFC(kTwoInvSqrtPi));
#pragma unroll
  for (int k = 1; k < DEG; ++k) {
    ar = df_sub(df_mul(zr, tr[k]), df_mul(y, ti[k]));
    ai = df_add(df_mul(zr, ti[k]), df_mul(y, tr[k]));
    const float s = -2.f / (float)(k + 1);  // exact for k + 1 in {2, 4}; else one rounding
    const F2 sc = (k + 1 == 3) ? F2(DFC(-2.0 / 3)) : (k + 1 == 5) ? F2(DFC(-2.0 / 5))
                                                                  : F2{s, 0.f};
    tr[k + 1] = df_mul(df_add(ar, tr[k - 1]), sc);
    ti[k + 1] = df_mul(df_add(ai, ti[k - 1]), sc);
  }
}

// FP64-accurate expansion: t_0, t_1 as pairs, t_2 .. t_5 in float (the width limits keep
// their rounding below 2e-13 of Re w).
struct TayP {
  F2 z0, t0r, t0i, t1r, t1i;
  float qr[4], qi[4];
};
__device__ __forceinline__ void tayp_from(TayP& T, F2 zr, const F2* tr, const F2* ti) {
  T.z0 = zr;
  T.t0r = tr[0];
  T.t0i = ti[0];
  T.t1r = tr[1];
  T.t1i = ti[1];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T.qr[k] = __fadd_rn(tr[k + 2].hi, tr[k + 2].lo);
    T.qi[k] = __fadd_rn(ti[k + 2].hi, ti[k + 2].lo);
  }
}
__device__ __forceinline__ void tayp_build(TayP& T, F2 zr, F2 y, const WeidCoef& W) {
  F2 tr[6], ti[6];
  tay_coefs<5>(zr, y, W, tr, ti);
  tayp_from(T, zr, tr, ti);
}
__device__ __forceinline__ void tayp_eval(const TayP& T, F2 zr, F2& wr, F2& wi) {
  const F2 dd = df_sub(zr, T.z0);
  const float d = dd.hi;
  const float qr = __fmaf_rn(__fmaf_rn(__fmaf_rn(T.qr[3], d, T.qr[2]), d, T.qr[1]), d, T.qr[0]);
  const float qi = __fmaf_rn(__fmaf_rn(__fmaf_rn(T.qi[3], d, T.qi[2]), d, T.qi[1]), d, T.qi[0]);
  wr = df_add(T.t0r, df_mul(dd, df_add_f(T.t1r, __fmul_rn(d, qr))));
  wi = df_add(T.t0i, df_mul(dd, df_add_f(T.t1i, __fmul_rn(d, qi))));
}

// ---- the table -----------------------------------------------------------------------------
// Entry j, kSBTabF4 float4: z0 (pair), t0r, t0i, t1r, t1i (pairs), qr[4], qi[4], and the
// cell's middle in x as a pair (x0 = mu + Re z0 / c1, the mixed plan's exact differences).

// The cell of an event with Re z ~ u (any float approximation: the cells' half-widths
// leave 4 % for a rounded u or logarithm).
struct SBTabF {
  int ntab, nneg, ncore;
  float a, ih, zc, izc, ilr;
};
__device__ __forceinline__ SBTabF sbtab_f(const SBTabHdr& H) {
  return SBTabF{H.ntab, H.nneg, H.ncore, H.a, H.ih, H.zc, H.izc, H.ilr};
}
__device__ __forceinline__ int sbtab_index(float u, const SBTabF& H) {
  int k;
  if (u < -H.zc) k = H.nneg - 1 - (int)(__logf(-u * H.izc) * H.ilr);
  else if (u < H.zc) k = H.nneg + (int)(fmaxf(u - H.a, 0.f) * H.ih);
  else k = H.nneg + H.ncore + (int)(__logf(u * H.izc) * H.ilr);
  return min(max(k, 0), H.ntab - 1);
}

// Middle of cell j (float: only its cell matters; the entry stores the value used).
__device__ __forceinline__ float sbtab_middle(int j, const SBTabHdr& H) {
  if (j < H.nneg) return -H.zc * __expf(((float)(H.nneg - 1 - j) + 0.5f) * H.lr);
  if (j < H.nneg + H.ncore) return __fmaf_rn((float)(j - H.nneg) + 0.5f, H.h, H.a);
  return H.zc * __expf(((float)(j - H.nneg - H.ncore) + 0.5f) * H.lr);
}

// Entry j: the expansion at the cell's middle, Re z0 = (x0 - mu) c1 formed as the events
// form Re z (x0 - mu exact in FP64, then pairs).
__device__ __forceinline__ void sbtab_build(int j, const SBTabHdr& H, const WeidCoef& W,
                                            float4* __restrict__ tab) {
  const double x0 = fma((double)sbtab_middle(j, H), H.ic1, H.mu);
  const F2 z0 = df_mul(df_split(x0 - H.mu), df_from(H.c1));
  F2 tr[6], ti[6];
  tay_coefs<5>(z0, df_from(H.y), W, tr, ti);
  TayP T;
  tayp_from(T, z0, tr, ti);
  const F2 xs = df_split(x0);
  float4* e = tab + (size_t)j * kSBTabF4;
  e[0] = make_float4(T.z0.hi, T.z0.lo, T.t0r.hi, T.t0r.lo);
  e[1] = make_float4(T.t0i.hi, T.t0i.lo, T.t1r.hi, T.t1r.lo);
  e[2] = make_float4(T.t1i.hi, T.t1i.lo, T.qr[0], T.qr[1]);
  e[3] = make_float4(T.qr[2], T.qr[3], T.qi[0], T.qi[1]);
  e[4] = make_float4(T.qi[2], T.qi[3], xs.hi, xs.lo);
}

// The FP64 plan's view of entry k.
__device__ __forceinline__ void sbtab_load(const float4* __restrict__ tab, int k, TayP& T) {
  const float4* e = tab + (size_t)k * kSBTabF4;
  const float4 a = __ldg(e), b = __ldg(e + 1), c = __ldg(e + 2), d = __ldg(e + 3),
               f = __ldg(e + 4);
  T.z0 = F2{a.x, a.y};
  T.t0r = F2{a.z, a.w};
  T.t0i = F2{b.x, b.y};
  T.t1r = F2{b.z, b.w};
  T.t1i = F2{c.x, c.y};
  T.qr[0] = c.z;
  T.qr[1] = c.w;
  T.qr[2] = d.x;
  T.qr[3] = d.y;
  T.qi[0] = d.z;
  T.qi[1] = d.w;
  T.qi[2] = f.x;
  T.qi[3] = f.y;
}

}  // namespace gfi
