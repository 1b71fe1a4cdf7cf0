// k_sigbkg.cu -- the event pass of a signal + background line-shape fit: an AddPdf of a
// Voigtian signal and a threshold background over one observable (Sec. 4: the D*+ width
// fit's line shape over the D*+ - D0 mass difference; Sec. 3: AddPdf), NLL and gradient.
//
// The general kernels (k_1d.cu) interpret the compiled program per event with the leaf
// constants and the gradient slots in shared memory.  This form holds everything in
// registers and takes the gradient from per-thread moments of the event sums:
//   NLL = -sum_i log P_i,   P = c_v V + c_t B,   V = c3 Re w(z),  z = (x - mu) c1 + i y,
//   dNLL/dtheta = -sum_i (dP_i/dtheta)/P_i,
// and with s = 1/P every derivative of V is a fixed linear combination (coefficients
// depending on theta only) of the sums
//   Ms = sum s, Mr = sum s Re w, Mi = sum s Im w, Mzr = sum s x_r Re w, Mzi = sum s x_r Im w,
//   Mzzr = sum s x_r^2 Re w   (x_r = Re z; w' = -2 z w + 2i/sqrt(pi)),
// every derivative of B one of  MB = sum s B, MtB = sum s t B, MBi = sum s B/t,
// MBl = sum s B log t  (t = x - x0), and the fraction's of Mr and MB.  The last block
// forms the gradient from the reduced moments in FP64.  The log-sum is a running product
// of the P_i with its binary exponent split off after every factor, whose logarithm is
// taken once per chunk of events.
//
// w(z) along the line Im z = y: every event reads its degree-5 Taylor expansion from the
// evaluation's table (sbtab.cuh), built by the normalisation launch at the middles of
// cells of Re z narrow enough for the expansion's validated limits, in any event order;
// the entry is reloaded only when an event's cell differs from the previous one's (sorted
// events in chunks mostly share one).  Without a table (a line too narrow for its cells
// to fit, y < 1e-6) w is expanded once per chunk of sorted events around the chunk's
// middle event, or evaluated per event by the Weideman series.
//
// Two arithmetics:
//  FP64 plan   double-float pairs on the FP32 pipe (as k_1d.cu): exact FP64 differences
//              x - mu, x - x0; the expansion's t_0, t_1 as pairs, t_2 .. t_5 in float;
//              events whose P leaves [2^-80, 2^125) are re-evaluated in FP64.
//  mixed plan  per-event arithmetic in FP32 (GF_MIXED): data enter by a bit split and exact
//              float differences (d = (x - x0) c1 from the cell middle's x0); the expansion
//              in float (its coefficients rounded from the FP64-accurate ones); the chunk's
//              moment sums in float, folded into pairs at the chunk's end; the log-sum, the
//              block and cross-block sums, the normalisation integrals (k_norm_1d) and the
//              gradient's combination in FP64-accurate arithmetic.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>

#include "devutil.cuh"
#include "gf_internal.h"
#include "launch.h"
#include "sbtab.cuh"

namespace gfi {
namespace {

// Threads per block: the FP64 plan one block of 512 per SM (128 registers a thread), the
// mixed plan two of 384 (80 registers); few blocks leave the last block one pass of loads
// for the cross-block sums (one value per warp).
template <bool MIXED>
__host__ __device__ constexpr int sb_threads() { return MIXED ? 384 : 512; }
template <bool MIXED>
__host__ __device__ constexpr int sb_min_blocks() { return MIXED ? 2 : 1; }
constexpr int kSBChunk64 = 48;     // FP64 plan: events per expansion of w, at most
constexpr int kSBSub64 = 8;        // ... and per sub-chunk of a chunk too wide for one
// FP64 plan: largest |Re z - Re z0| of an expanded chunk.  The float coefficients t2..t5
// set the error, 6e-8 |t2| d^2 relative; measured against a 30-digit w over |Re z0| <= 6:
// at d = 3e-4 below 1.1e-13 of Re w for every y in 1e-4 .. 1, at d = 6e-4 below 1.7e-13
// for y >= 0.03 (4.4e-13 at y = 1e-3, where the Gaussian part's steep derivatives set
// |t2/t0| up to ~20 near |Re z| = 2.5)
constexpr float kSBLim64 = 3e-4f;
constexpr float kSBLim64W = 6e-4f;
constexpr double kSBLim64WY = 0.03;
// FP64 plan, |Re z0| >= 6 and y >= 1e-6: the limit kSBLim64Rel |Re z0|.  There Re w is the
// Lorentzian tail (the Gaussian part exp(-x^2) <= 2.3e-16 is below 1e-8 of it), whose
// Taylor coefficients on the real line fall as |Re t_k| ~ (k + 1) Re w / |x|^k: with
// d = rho |x| the float coefficients t2..t5 carry a relative error of 6e-8 x 3 rho^2
// (9.5e-14 measured at rho = 5e-4 against a 30-digit w, y = 1e-3 .. 1, |x| = 6 .. 40) and
// the truncation 7 rho^6 (1e-19)
constexpr float kSBLim64Rel = 5e-4f;
constexpr int kSBChunk32 = 96;     // mixed plan
constexpr int kSBSub32 = 24;
// mixed plan: largest |Re z - Re z0| at |Re z0| < 0.6 (the Cauchy bound |t_k| <= 6 on the
// unit circle around z0: degree-4 truncation below 6 d^5 ~ 1.5e-12), and a wider one,
// 0.005 |Re z0|, for |z0| >= 2, where |w| <= 1.2/|z0| on the circle of radius |z0|/2
// gives |t_k| <= (1.2/|z0|)(2/|z0|)^k and a truncation below 1.2/|z0| (0.01)^5, i.e.
// 2e-9 |z0| relative to Re w >= 0.05 y/|z0|^2 (y = 0.094 here): FP32-level
constexpr float kSBLim32 = 3e-3f;
constexpr float kSBLim32Rel = 5e-3f;
constexpr int kSBFlush = 32;       // unsorted loop: events per log of the running product
constexpr int kSBMom = 11;         // reduced values: sum log P and ten moments

enum { SB_LOGP = 0, SB_S, SB_R, SB_I, SB_ZR, SB_ZI, SB_ZZR, SB_B, SB_TB, SB_BI, SB_BL };

// ---- running product of P with its exponent split off -------------------------------------
struct ProdF2 {
  F2 p = {1.f, 0.f};
  int e = 0;
  __device__ __forceinline__ void mul(F2 x) {
    p = df_mul(p, x);
    const int k = (int)((__float_as_uint(p.hi) >> 23) & 0xff) - 127;
    const float sc = __uint_as_float((unsigned)(127 - k) << 23);  // 2^-k, exact
    p.hi = __fmul_rn(p.hi, sc);
    p.lo = __fmul_rn(p.lo, sc);
    e += k;
  }
  // log of the product (the caller resets it)
  __device__ __forceinline__ F2 log() const {
    constexpr DFC ln2(0.69314718055994530942);
    return df_add(df_log_tab(p, s_log_tab), df_mul_f(F2(ln2), (float)e));
  }
};
struct ProdF {
  float p = 1.f;
  int e = 0;
  __device__ __forceinline__ void mul(float x) {
    p = __fmul_rn(p, x);
    const int k = (int)((__float_as_uint(p) >> 23) & 0xff) - 127;
    p = __fmul_rn(p, __uint_as_float((unsigned)(127 - k) << 23));
    e += k;
  }
  __device__ __forceinline__ F2 log() const {
    constexpr DFC ln2(0.69314718055994530942);
    return df_add(df_log_tab(F2{p, 0.f}, s_log_tab), df_mul_f(F2(ln2), (float)e));
  }
};

// Pair sum whose low part is renormalised only on demand (sums of a few dozen terms).
struct Lazy {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(F2 v) {
    const F2 s = two_sum(hi, v.hi);
    hi = s.hi;
    lo = __fadd_rn(lo, __fadd_rn(s.lo, v.lo));
  }
  __device__ __forceinline__ void norm() {
    const F2 s = fast_two_sum(hi, lo);
    hi = s.hi;
    lo = s.lo;
  }
  __device__ __forceinline__ F2 get() const { return fast_two_sum(hi, lo); }
};

// Weideman's series in float (the mixed plan's unsorted events and wide chunks): the same
// coefficients and rational map as faddeeva_f2, every step in FP32.
__device__ __forceinline__ void faddeeva_f32(float x, float y, const WeidCoef& W, float& wr,
                                             float& wi) {
  const float L = W.Lhi;
  const float dr = L + y;                     // L - iz = dr - i x
  const float inv = 1.f / __fmaf_rn(dr, dr, x * x);
  const float zr = __fmaf_rn(L - y, dr, -x * x) * inv;
  const float zi = 2.f * L * x * inv;
  float pr = W.ahi[kWeidN], pi = 0.f;
#pragma unroll 8
  for (int n = kWeidN - 1; n >= 1; --n) {
    const float t = __fmaf_rn(pr, zr, __fmaf_rn(-pi, zi, W.ahi[n]));
    pi = __fmaf_rn(pr, zi, pi * zr);
    pr = t;
  }
  const float ir = dr * inv, ii = x * inv;   // 1/(L - iz)
  const float qr = __fmaf_rn(ir, ir, -ii * ii), qi = 2.f * ir * ii;
  wr = __fmaf_rn(0.56418958354775628695f, ir, 2.f * __fmaf_rn(pr, qr, -pi * qi));
  wi = __fmaf_rn(0.56418958354775628695f, ii, 2.f * __fmaf_rn(pr, qi, pi * qr));
}

// The mixed plan's direct evaluation out of line: inline, its code would be repeated in
// every unrolled copy of the event body.  (The FP64 plan keeps its direct path inline: its
// event loop is not unrolled, and a call would save and restore the live pairs.)
__device__ __noinline__ void w_direct_f32(float x, float y, const WeidCoef& W, float& wr,
                                          float& wi) {
  faddeeva_f32(x, y, W, wr, wi);
}

// ---- constants of one evaluation -------------------------------------------------------------
// From the leaf records (k_norm_1d): Voigtian c0 = mu, c1 = 1/(sigma sqrt2), c2 = y = Im z,
// c3 = 1/(sigma sqrt(2 pi) N); threshold c0 = x0, c1 = p, c2 = c, c3 = 1/N.
struct SBConst {
  double mu, x0, c1, y, c3v, pw, cc, c3t, cv, ct;
  // the mixed plan's split P = ref (ca Re w + cb t^p e^{-c t}), ref > 0 (0: P = 0), one of
  // ca, cb exactly 1: every constant that scales all events stays in FP64 (ref and its log
  // enter the sums once per chunk), so FP32 rounding leaves no theta-dependent bias common
  // to all events
  double ref, lref, ca, cb;
  int half;  // p == 1/2 and no gradient in p: sqrt(t) instead of exp(p log t)
};
template <bool MIXED>
__device__ __forceinline__ void sb_consts(const SigBkgDesc& D, const double* __restrict__ der,
                                          bool grad, SBConst& K) {
  const double* rv = der + D.slot_v * kLeafRec;
  const double* rt = der + D.slot_t * kLeafRec;
  K.mu = rv[10];
  K.c1 = rv[11];
  K.y = rv[12];
  K.c3v = rv[13];
  K.x0 = rt[10];
  K.pw = rt[11];
  K.cc = rt[12];
  K.c3t = rt[13];
  K.cv = der[kMaxLeaf * kLeafRec + D.cslot_v];
  K.ct = der[kMaxLeaf * kLeafRec + D.cslot_t];
  K.half = (K.pw == 0.5 && !(grad && D.gt[1] >= 0)) ? 1 : 0;
  if (!MIXED) return;  // the split below is the mixed plan's
  const double kv = K.cv * K.c3v, kt = K.ct * K.c3t;
  double ref = fabs(kv) >= fabs(kt) ? kv : kt;
  K.ca = ref != 0.0 ? kv / ref : 0.0;
  K.cb = ref != 0.0 ? kt / ref : 0.0;
  if (ref < 0.0) {
    ref = -ref;
    K.ca = -K.ca;
    K.cb = -K.cb;
  }
  K.ref = ref;
  K.lref = log(ref);
}

// One event in FP64 (P outside the float-safe range): log P and the moments' terms.
__device__ __noinline__ void sb_event_fp64(double x, const SBConst* __restrict__ K,
                                           const WeidCoef& W, double* o) {
  const double zr = (x - K->mu) * K->c1;
  double wr, wi;
  faddeeva_df(zr, K->y, W, wr, wi);
  const double V = K->c3v * wr;
  const double t = x - K->x0;
  double B = 0.0, lt = 0.0;
  if (t > 0.0) {
    lt = df_log(t);
    B = df_exp(K->pw * lt - K->cc * t) * K->c3t;
  }
  const double P = K->cv * V + K->ct * B;
  const double s = 1.0 / P;
  o[SB_LOGP] = df_log(P);
  o[SB_S] = s;
  o[SB_R] = s * wr;
  o[SB_I] = s * wi;
  o[SB_ZR] = zr * s * wr;
  o[SB_ZI] = zr * s * wi;
  o[SB_ZZR] = zr * zr * s * wr;
  o[SB_B] = s * B;
  o[SB_TB] = t > 0.0 ? s * B * t : 0.0;
  o[SB_BI] = t > 0.0 ? s * B / t : 0.0;
  o[SB_BL] = t > 0.0 ? s * B * lt : 0.0;
}

// Last block: NLL and gradient from the reduced sums M (FP64) into result[0 .. nfree].
__device__ void sb_finish(const SigBkgDesc& D, const double* __restrict__ der, const double* M,
                          bool grad, double* __restrict__ result) {
  result[0] = -M[SB_LOGP];
  if (!grad) return;
  double g[kMaxFree1D];
  for (int k = 0; k < D.nfree; ++k) g[k] = 0.0;
  const double* rv = der + D.slot_v * kLeafRec;
  const double* rt = der + D.slot_t * kLeafRec;
  const double cv = der[kMaxLeaf * kLeafRec + D.cslot_v];
  const double ct = der[kMaxLeaf * kLeafRec + D.cslot_t];
  const double y = rv[12], c3 = rv[13];
  // sums of s dRe w/dx_r, s dIm w/dx_r and s (dRe w/dx_r x_r - dIm w/dx_r y)
  const double s_dre = -2.0 * (M[SB_ZR] - y * M[SB_I]);
  const double s_dim = -2.0 * (M[SB_ZI] + y * M[SB_R]) + kTwoInvSqrtPi * M[SB_S];
  const double s_q = -2.0 * M[SB_ZZR] + 4.0 * y * M[SB_ZI] + 2.0 * y * y * M[SB_R] -
                     kTwoInvSqrtPi * y * M[SB_S];
  const double sv = c3 * M[SB_R];  // sum V/P
  // Voigtian: dV/dmu = -(c5 dre + V r2), dV/dsigma = -(c6 q + V c8), dV/dGamma = -(c7 dim
  // + V r4), c5..c8 = rec[15..18], r_k = dlogN/dpar = rec[2..4]
  if (D.gv[0] >= 0) g[D.gv[0]] += cv * (rv[15] * s_dre + rv[2] * sv);
  if (D.gv[1] >= 0) g[D.gv[1]] += cv * (rv[16] * s_q + rv[18] * sv);
  if (D.gv[2] >= 0) g[D.gv[2]] += cv * (rv[17] * s_dim + rv[4] * sv);
  // threshold: dB/dx0 = B (c - p/t - r2), dB/dp = B (log t - r3), dB/dc = -B (t + r4)
  if (D.gt[0] >= 0) g[D.gt[0]] -= ct * ((rt[12] - rt[2]) * M[SB_B] - rt[11] * M[SB_BI]);
  if (D.gt[1] >= 0) g[D.gt[1]] -= ct * (M[SB_BL] - rt[3] * M[SB_B]);
  if (D.gt[2] >= 0) g[D.gt[2]] += ct * (M[SB_TB] + rt[4] * M[SB_B]);
  // fractions: dP/df = +-V or +-B
  if (D.fpos_v >= 0) g[D.fpos_v] -= D.fsgn_v * sv;
  if (D.fpos_t >= 0) g[D.fpos_t] -= D.fsgn_t * M[SB_B];
  for (int k = 0; k < D.nfree; ++k) result[1 + k] = g[k];
}

// ---- the kernel -------------------------------------------------------------------------------
// STORE: log P_i into out_logp[perm ? perm[i] : i] instead of the sums.
// Shared scratch of one block.
template <bool MIXED>
struct SBShared {
  static constexpr int NT = sb_threads<MIXED>();
  static constexpr int NM = MIXED ? kSBMom - 1 : 1;
  SBConst K;
  // mixed plan: the per-thread pair sums of the moments (touched once per chunk) and the
  // constants used only at chunk boundaries, as pairs, out of the registers
  float mh[NM][MIXED ? NT : 1], ml[NM][MIXED ? NT : 1];
  F2 mu2, yp, sv, st, lref;
  F2 kp[8];    // the per-event constants as pairs (warp 0 converts them, one per lane)
  SBTabF tf;   // the table of w expansions (tf.ntab = 0: none)
  WeidCoef W;  // the series coefficients, read by every thread (and the out-of-line paths)
  double red[(NT / 32) * kSBMom > NT ? (NT / 32) * kSBMom : NT];  // block sums; NT pairs for
                                                                   // the cross-block sums
  double fin[kSBMom];
  int last;
};

// The sorted events cut into nch = J T chunks (T threads, J = ceil(n / (T cmax))) of
// floor(n / nch) or that plus one events, so that every thread walks exactly J chunks and
// the same number of events to within J; chunk c starts at q c + floor(r c / nch) for
// n = q nch + r (r c < nch^2: no overflow below 3 x 10^9 chunks).
struct ChunkSplit {
  int64_t nch, q, r;
  __device__ ChunkSplit(int64_t n, int64_t nthreads, int cmax) {
    const int64_t per = nthreads * cmax;
    nch = (n + per - 1) / per * nthreads;
    q = n / nch;
    r = n - q * nch;
  }
  __device__ int64_t start(int64_t c) const { return q * c + r * c / nch; }
};

// Body of one (virtual) block vb of a launch of vgrid blocks over one data set; the last
// block to arrive finishes the reduction.  sorted: the events are sorted ascending by x.
template <bool G, bool MIXED, bool STORE>
__device__ __forceinline__ void sigbkg_block(
    const SigBkgDesc& D, const WeidCoef& Wg, const int sorted, const double* __restrict__ xcol,
    const int64_t n, const double* __restrict__ der, double* __restrict__ partials,
    unsigned* __restrict__ counter, double* __restrict__ result, double* __restrict__ out_logp,
    const int32_t* __restrict__ perm, const SBTabHdr* __restrict__ tabh,
    const float4* __restrict__ tab, const int vb, const int vgrid, SBShared<MIXED>& sh) {
  const int tid = threadIdx.x;
  constexpr int NT = sb_threads<MIXED>();
  const int64_t nthreads = (int64_t)vgrid * NT;
  // sorted events and at least 8 per thread: one expansion of w per chunk pays
  const bool chunked = sorted && n >= 8 * nthreads;
  if (tid == 0) {
    sb_consts<MIXED>(D, der, G, sh.K);
    sh.tf = tab && !chunked ? sbtab_f(*tabh) : SBTabF{0, 0, 0, 0.f, 0.f, 0.f, 0.f, 0.f};
  }
  // the constants as pairs, one per lane of warp 0 (their FP64 conversions and divisions
  // side by side instead of in a chain on one thread or repeated by every thread)
  if (tid < 32) {
    __syncwarp();
    const SBConst& k = sh.K;
    if constexpr (!MIXED) {
      if (tid < 8) {
        const double v = tid == 0 ? k.c1 : tid == 1 ? k.y : tid == 2 ? k.c3v : tid == 3 ? k.pw
                       : tid == 4 ? k.cc : tid == 5 ? k.c3t : tid == 6 ? k.cv : k.ct;
        sh.kp[tid] = df_from(v);
      }
    } else {
      switch (tid) {
        case 0: sh.mu2 = df_split(k.mu); break;
        case 1: sh.yp = df_from(k.y); break;
        case 2: sh.sv = df_from(1.0 / k.ref); break;
        case 3: sh.st = df_from(k.c3t / k.ref); break;
        case 4: sh.lref = df_from(k.lref); break;
        case 5: sh.kp[0] = df_from(k.c1); break;
        case 6: sh.kp[1] = df_from(k.cc); break;
        case 7: sh.kp[2] = df_from(k.pw); break;
        case 8: sh.kp[3] = df_from(k.ca); break;
        case 9: sh.kp[4] = df_from(k.cb); break;
        case 10: sh.kp[5] = df_split(k.x0); break;
        default: break;
      }
    }
  }
  if constexpr (MIXED && G)
    for (int k = 0; k < kSBMom - 1; ++k) sh.mh[k][tid] = sh.ml[k][tid] = 0.f;
  {
    const float* src = reinterpret_cast<const float*>(&Wg);
    float* dst = reinterpret_cast<float*>(&sh.W);
    for (int k = tid; k < (int)(sizeof(WeidCoef) / sizeof(float)); k += blockDim.x) dst[k] = src[k];
  }
  __syncthreads();
  const SBConst& K = sh.K;
  // the series coefficients: the kernel parameter (constant bank) for the inline paths, the
  // shared copy for the mixed plan's out-of-line direct path
  const WeidCoef& W = Wg;
  const WeidCoef& Ws = sh.W;

  Lazy acc;            // sum log P
  Lazy m[kSBMom - 1];  // moments SB_S .. SB_BL
  const bool need_bi = G && D.gt[0] >= 0;
  const bool need_bl = G && D.gt[1] >= 0;
  const bool half = K.half != 0;

  // FP64 fallback for one event (P outside the float-safe range or not positive)
  auto fallback = [&](int64_t i, double xi) {
    double o[kSBMom];
    sb_event_fp64(xi, &K, Ws, o);
    if (STORE) {
      out_logp[perm ? perm[i] : i] = o[SB_LOGP];
      return;
    }
    acc.add(df_from(o[SB_LOGP]));
    if (G)
#pragma unroll
      for (int k = 1; k < kSBMom; ++k) m[k - 1].add(df_from(o[k]));
  };

  const int64_t g = (int64_t)vb * NT + tid;
  constexpr int kChunk = MIXED ? kSBChunk32 : kSBChunk64;
  (void)g;

  // the table of w expansions for events in any order: each event's expansion by its cell
  // of Re z, reloaded when the cell changes.  Sorted chunks expand w themselves (one
  // Weideman series and recurrence per chunk costs less than a cell lookup per event).
  const bool use_tab = sh.tf.ntab > 0;  // (never in chunks)
  int kcur = -1;

  if constexpr (!MIXED) {
    // ---------------- FP64 plan: pairs ----------------
    const F2 c1 = sh.kp[0], y = sh.kp[1], c3v = sh.kp[2];
    const F2 pw = sh.kp[3], cc = sh.kp[4], c3t = sh.kp[5];
    const F2 cv = sh.kp[6], ct = sh.kp[7];
    ProdF2 prod;
    TayP T;
    // tabc: std::true_type for the table's lookups, std::false_type for the chunk's own
    // expansion (tay) or the series (the two loops get their own code)
    auto one = [&](int64_t i, double xi, bool tay, auto tabc) {
      const F2 zr = df_mul(df_split(xi - K.mu), c1);
      F2 wr, wi;
      if constexpr (decltype(tabc)::value) {
        const int kc = sbtab_index(zr.hi, sh.tf);
        if (kc != kcur) {
          sbtab_load(tab, kc, T);
          kcur = kc;
        }
        tayp_eval(T, zr, wr, wi);
      } else if (tay) {
        tayp_eval(T, zr, wr, wi);
      } else {
        faddeeva_f2(zr, y, W, wr, wi);
      }
      const double td = xi - K.x0;
      F2 B = {0.f, 0.f}, t = {0.f, 0.f}, lt = {0.f, 0.f};
      if (td > 0.0) {
        t = df_split(td);
        if (half) {
          B = df_mul(df_mul(df_sqrt(t), df_exp_tab(df_neg(df_mul(cc, t)), s_exp_tab)), c3t);
        } else {
          lt = df_log_tab(t, s_log_tab);
          B = df_mul(df_exp_tab(df_sub(df_mul(pw, lt), df_mul(cc, t)), s_exp_tab), c3t);
        }
      }
      const F2 P = df_add(df_mul(cv, df_mul(c3v, wr)), df_mul(ct, B));
      if (!(P.hi >= 8.271806125530277e-25f && P.hi < 4.2535295865117308e37f)) {
        fallback(i, xi);
        return;
      }
      if (STORE) {
        out_logp[perm ? perm[i] : i] = df_to(df_log_tab(P, s_log_tab));
        return;
      }
      prod.mul(P);
      if (G) {
        const F2 s = df_rcp(P);
        const F2 a = df_mul(s, wr), b = df_mul(s, wi);
        const F2 za = df_mul(zr, a);
        m[SB_S - 1].add(s);
        m[SB_R - 1].add(a);
        m[SB_I - 1].add(b);
        m[SB_ZR - 1].add(za);
        m[SB_ZI - 1].add(df_mul(zr, b));
        m[SB_ZZR - 1].add(df_mul(zr, za));
        if (td > 0.0) {
          const F2 sb = df_mul(s, B);
          m[SB_B - 1].add(sb);
          m[SB_TB - 1].add(df_mul(t, sb));
          if (need_bi) m[SB_BI - 1].add(df_mul(sb, df_rcp(t)));
          if (need_bl) m[SB_BL - 1].add(df_mul(sb, lt));
        }
      }
    };
    auto flush = [&]() {
      if (STORE) return;
      acc.add(prod.log());
      prod = ProdF2();
      acc.norm();
      if (G)
#pragma unroll
        for (int k = 0; k < kSBMom - 1; ++k) m[k].norm();
    };
    if (chunked) {
      // the sorted events in chunks of at most kChunk (ChunkSplit) with one expansion of w
      // per chunk; chunk c
      // goes to the thread of index c mod T in block-cyclic order (thread t of block b
      // takes c = j T + t B + b), so that the consecutive chunks of a region that costs
      // more -- a sparse edge of the data, where a chunk too wide for one expansion is
      // taken as sub-chunks of kSBSub64 and a sub-chunk still too wide evaluates w per
      // event -- spread over all blocks instead of loading a few SMs
      const int64_t gc = (int64_t)tid * vgrid + vb;
      const bool wide_ok = K.y >= 1e-6;
      const float lim0 = K.y >= kSBLim64WY ? kSBLim64W : kSBLim64;
      auto expand = [&](int64_t a, int c) {  // expansion for events a .. a + c - 1, if narrow
        const double xm = __ldg(xcol + a + (c - 1) / 2);
        const float da = fabsf(__fmul_rn((float)(__ldg(xcol + a) - xm), c1.hi));
        const float db = fabsf(__fmul_rn((float)(__ldg(xcol + a + c - 1) - xm), c1.hi));
        const float az = fabsf(__fmul_rn((float)(xm - K.mu), c1.hi));
        const float lim = wide_ok && az >= 6.f ? fmaxf(lim0, kSBLim64Rel * az) : lim0;
        const bool ok = fmaxf(da, db) <= lim;
        if (ok) tayp_build(T, df_mul(df_split(xm - K.mu), c1), y, W);
        return ok;
      };
      auto run = [&](int64_t a, int c, bool tay) {  // the next event's load in flight
        double xn = __ldg(xcol + a);
        for (int k = 0; k < c; ++k) {
          const double xi = xn;
          if (k + 1 < c) xn = __ldg(xcol + a + k + 1);
          one(a + k, xi, tay, std::false_type{});
        }
      };
      const ChunkSplit cs(n, nthreads, kChunk);
      for (int64_t ci = gc; ci < cs.nch; ci += nthreads) {
        const int64_t c0 = cs.start(ci);
        const int cnt = (int)(cs.start(ci + 1) - c0);
        if (expand(c0, cnt)) {
          run(c0, cnt, true);
        } else {
          for (int s0 = 0; s0 < cnt; s0 += kSBSub64) {
            const int sc = cnt - s0 < kSBSub64 ? cnt - s0 : kSBSub64;
            run(c0 + s0, sc, expand(c0 + s0, sc));
          }
        }
        flush();
      }
    } else {
      auto loop = [&](auto tabc) {
        int since = 0;
        for (int64_t i = g; i < n; i += nthreads) {
          one(i, __ldcs(xcol + i), false, tabc);
          if (++since == kSBFlush) {
            flush();
            since = 0;
          }
        }
        flush();
      };
      if (use_tab) loop(std::true_type{});
      else loop(std::false_type{});
    }
  } else {
    // ---------------- mixed plan: FP32 per event ----------------
    const F2 x02 = sh.kp[5];
    const float y = sh.yp.hi;
    // constants that multiply per-event values as pairs (one extra FMA each): the float
    // result then carries per-event rounding only
    const F2 c1p = sh.kp[0], ccp = sh.kp[1], pwp = sh.kp[2];
    const F2 cap = sh.kp[3], cbp = sh.kp[4];
    auto kmul = [](float a, F2 c) { return __fmaf_rn(a, c.hi, __fmul_rn(a, c.lo)); };
    ProdF prod;
    int pcount = 0;  // events in the running product
    float cm[kSBMom - 1];
#pragma unroll
    for (int k = 0; k < kSBMom - 1; ++k) cm[k] = 0.f;
    // one event: x as a pair, zr = Re z, dz = Re z - Re z0 (tay: T holds the expansion's
    // coefficients to degree 5, re then im (a chunk's own expansion: degree 4, the table's:
    // 5); otherwise the float series)
    float T[12] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    auto one = [&](int64_t i, double xi, F2 xs, float zr, float dz, bool tay) {
      float wr, wi;
      if (tay) {
        wr = __fmaf_rn(__fmaf_rn(__fmaf_rn(__fmaf_rn(__fmaf_rn(T[5], dz, T[4]), dz, T[3]), dz, T[2]), dz,
                                 T[1]), dz, T[0]);
        wi = __fmaf_rn(__fmaf_rn(__fmaf_rn(__fmaf_rn(__fmaf_rn(T[11], dz, T[10]), dz, T[9]), dz, T[8]),
                                 dz, T[7]), dz, T[6]);
      } else {
        w_direct_f32(zr, y, Ws, wr, wi);
      }
      const float t = __fadd_rn(__fsub_rn(xs.hi, x02.hi), __fsub_rn(xs.lo, x02.lo));
      float B = 0.f, lt = 0.f;
      if (t > 0.f) {
        if (half) {
          B = __fmul_rn(__fmul_rn(t, rsqrtf(t)), __expf(-kmul(t, ccp)));
        } else {
          lt = __logf(t);
          B = __expf(kmul(lt, pwp) - kmul(t, ccp));
        }
      }
      const float P = __fadd_rn(kmul(wr, cap), kmul(B, cbp));  // P / ref
      if (!(P >= 8.271806125530277e-25f && P < 4.2535295865117308e37f)) {
        fallback(i, xi);
        return;
      }
      if (STORE) {
        out_logp[perm ? perm[i] : i] = (double)logf(P) + K.lref;
        return;
      }
      prod.mul(P);
      ++pcount;
      if (G) {
        const float s = __fdividef(1.f, P);
        const float a = s * wr, b = s * wi, za = zr * a;
        cm[SB_S - 1] += s;
        cm[SB_R - 1] += a;
        cm[SB_I - 1] += b;
        cm[SB_ZR - 1] += za;
        cm[SB_ZI - 1] += zr * b;
        cm[SB_ZZR - 1] += zr * za;
        if (t > 0.f) {
          const float sb = s * B;
          cm[SB_B - 1] += sb;
          cm[SB_TB - 1] += t * sb;
          if (need_bi) cm[SB_BI - 1] += __fdividef(sb, t);
          if (need_bl) cm[SB_BL - 1] += sb * lt;
        }
      }
    };
    // chunk end: log of the product plus its events' log(ref); the float sums of the chunk
    // in units of 1/ref (Voigtian terms) and c3t/ref (background terms) folded into pairs
    auto flush = [&]() {
      if (STORE) return;
      acc.add(prod.log());
      if (pcount) acc.add(df_mul_f(sh.lref, (float)pcount));
      prod = ProdF();
      pcount = 0;
      acc.norm();
      if (G) {
        const F2 sv = sh.sv, st = sh.st;
#pragma unroll
        for (int k = 0; k < kSBMom - 1; ++k) {
          const F2 v = df_mul_f(k + 1 < SB_B ? sv : st, cm[k]);
          const F2 a = two_sum(sh.mh[k][tid], v.hi);
          sh.mh[k][tid] = a.hi;
          const F2 b = fast_two_sum(a.hi, __fadd_rn(sh.ml[k][tid], __fadd_rn(a.lo, v.lo)));
          sh.mh[k][tid] = b.hi;
          sh.ml[k][tid] = b.lo;
          cm[k] = 0.f;
        }
      }
    };
    // the current expansion's middle: x as a pair, Re z in float
    F2 xms = {0.f, 0.f};
    float z0f = 0.f;
    auto dzof = [&](F2 xs) {
      return kmul(__fadd_rn(__fsub_rn(xs.hi, xms.hi), __fsub_rn(xs.lo, xms.lo)), c1p);
    };
    // table entry kc as the float expansion around its cell's middle
    auto mload = [&](int kc) {
      const float4* e = tab + (size_t)kc * kSBTabF4;
      const float4 a = __ldg(e), b = __ldg(e + 1), c = __ldg(e + 2), d = __ldg(e + 3),
                   f = __ldg(e + 4);
      z0f = __fadd_rn(a.x, a.y);
      T[0] = __fadd_rn(a.z, a.w);
      T[1] = __fadd_rn(b.z, b.w);
      T[2] = c.z;
      T[3] = c.w;
      T[4] = d.x;
      T[5] = d.y;
      T[6] = __fadd_rn(b.x, b.y);
      T[7] = __fadd_rn(c.x, c.y);
      T[8] = d.z;
      T[9] = d.w;
      T[10] = f.x;
      T[11] = f.y;
      xms = F2{f.z, f.w};
      kcur = kc;
    };
    if (use_tab) mload(0);
    // an event's dz in the table: z0f + dz approximates Re z from any entry, and picks the
    // cell whose entry then serves the event
    auto tdz = [&](F2 xs) {
      float dz = dzof(xs);
      const int kc = sbtab_index(__fadd_rn(z0f, dz), sh.tf);
      if (kc != kcur) {
        mload(kc);
        dz = dzof(xs);
      }
      return dz;
    };
    if (chunked) {
      // chunks distributed over the threads as in the FP64 plan
      const int64_t gc = (int64_t)tid * vgrid + vb;
      // expansion (degree 4, float coefficients from the pair series) for events a ..
      // a + c - 1 when they lie close enough to the middle one
      auto expand = [&](int64_t a, int c) {
        const double xm = __ldg(xcol + a + (c - 1) / 2);
        xms = df_split(xm);
        const F2 z0 = df_mul(df_split(xm - K.mu), c1p);  // (Re z0 in pairs)
        z0f = __fadd_rn(z0.hi, z0.lo);
        const float da = fabsf(dzof(df_split(__ldg(xcol + a))));
        const float db = fabsf(dzof(df_split(__ldg(xcol + a + c - 1))));
        const float az = fabsf(z0f);
        const bool ok = fmaxf(da, db) <= (az >= 2.f ? fmaxf(kSBLim32, kSBLim32Rel * az) : kSBLim32);
        if (ok) {
          F2 tr[5], ti[5];
          tay_coefs<4>(z0, sh.yp, W, tr, ti);
#pragma unroll
          for (int k = 0; k < 5; ++k) {
            T[k] = __fadd_rn(tr[k].hi, tr[k].lo);
            T[6 + k] = __fadd_rn(ti[k].hi, ti[k].lo);
          }
        }
        return ok;
      };
      auto run = [&](int64_t a, int c, bool tay) {  // the loads of 4 events in flight at once
        for (int k = 0; k < c; k += 4) {
          double xv[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) xv[j] = k + j < c ? __ldg(xcol + a + k + j) : 0.0;
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (k + j < c) {
              const F2 xs = df_split(xv[j]);
              if (tay) {
                const float dz = dzof(xs);
                one(a + k + j, xv[j], xs, __fadd_rn(z0f, dz), dz, true);
              } else {
                const F2 mu2 = sh.mu2;
                const float zr =
                    kmul(__fadd_rn(__fsub_rn(xs.hi, mu2.hi), __fsub_rn(xs.lo, mu2.lo)), c1p);
                one(a + k + j, xv[j], xs, zr, 0.f, false);
              }
            }
        }
      };
      const ChunkSplit cs(n, nthreads, kChunk);
      for (int64_t ci = gc; ci < cs.nch; ci += nthreads) {
        const int64_t c0 = cs.start(ci);
        const int cnt = (int)(cs.start(ci + 1) - c0);
        if (expand(c0, cnt)) {
          run(c0, cnt, true);
        } else {
          for (int s0 = 0; s0 < cnt; s0 += kSBSub32) {
            const int sc = cnt - s0 < kSBSub32 ? cnt - s0 : kSBSub32;
            run(c0 + s0, sc, expand(c0 + s0, sc));
          }
        }
        flush();
      }
    } else {
      int since = 0;
      for (int64_t i = g; i < n; i += nthreads) {
        const double xi = __ldcs(xcol + i);
        const F2 xs = df_split(xi);
        if (use_tab) {
          const float dz = tdz(xs);
          one(i, xi, xs, __fadd_rn(z0f, dz), dz, true);
        } else {
          const F2 mu2 = sh.mu2;
          const float zr =
              kmul(__fadd_rn(__fsub_rn(xs.hi, mu2.hi), __fsub_rn(xs.lo, mu2.lo)), c1p);
          one(i, xi, xs, zr, 0.f, false);
        }
        if (++since == kSBChunk32) {
          flush();
          since = 0;
        }
      }
      flush();
    }
  }
  if (STORE) return;

  // block sums (fixed order), then the last block's cross-block sums and the gradient
  const int mm = G ? kSBMom : 1;
  F2 vals[kSBMom];  // the register (FP64 plan) or shared (mixed plan) sums, copied once
  vals[0] = acc.get();
#pragma unroll
  for (int k = 1; k < kSBMom; ++k)
    if constexpr (MIXED) vals[k] = F2{sh.mh[k - 1][tid], sh.ml[k - 1][tid]};
    else vals[k] = m[k - 1].get();
  // partials padded block-major: value k of block b at partials[b partial_stride(mm) + k]
  block_sum_pairs<G ? kSBMom : 1>([&](int k) -> F2 { return vals[k]; }, mm, sh.red,
                                  partials + (size_t)vb * partial_stride(mm), 1);
  if (!arrive_last_of(counter, (unsigned)vgrid, &sh.last)) return;
  reduce_partials_bm(partials, vgrid, mm, sh.fin, reinterpret_cast<F2*>(sh.red));
  if (tid == 0) {
    sb_finish(D, der, sh.fin, G, result);
    *counter = 0u;
  }
}

template <bool G, bool MIXED, bool STORE>
__global__ void __launch_bounds__(sb_threads<MIXED>(), sb_min_blocks<MIXED>()) k_sigbkg(
    const __grid_constant__ SigBkgDesc D, const __grid_constant__ WeidCoef W,
    const Program* __restrict__ prog, const double* __restrict__ xcol, const int64_t n,
    const double* __restrict__ der, double* __restrict__ partials,
    unsigned* __restrict__ counter, double* __restrict__ result, double* __restrict__ out_logp,
    const int32_t* __restrict__ perm, const SBTabHdr* __restrict__ tabh,
    const float4* __restrict__ tab) {
  __shared__ SBShared<MIXED> sh;
  load_df_tables();  // visible after the block body's first barrier
  sigbkg_block<G, MIXED, STORE>(D, W, prog->sorted, xcol, n, der, partials, counter, result,
                                out_logp, perm, tabh, tab, blockIdx.x, gridDim.x, sh);
}

// The fit server's batched tick: every waiting signal + background fit in one persistent
// launch; item it of the work list is virtual block it - item0 of its fit, which processes
// the events of the fit's standalone block of that index (the same bits alone or batched).
template <bool MIXED>
__global__ void __launch_bounds__(sb_threads<MIXED>(), sb_min_blocks<MIXED>())
    k_tick_sigbkg(const TickItem* __restrict__ items, int nfits, int total,
                  const __grid_constant__ WeidCoef W) {
  __shared__ SBShared<MIXED> sh;
  load_df_tables();
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    int f = 0;
    while (f + 1 < nfits && items[f + 1].item0 <= it) ++f;
    const TickItem& ti = items[f];
    const FitSB* F = static_cast<const FitSB*>(ti.fit);
    sigbkg_block<true, MIXED, false>(F->D, W, F->sorted, F->x, F->n, F->derived, F->partials,
                                     F->counter, ti.result, nullptr, nullptr,
                                     reinterpret_cast<const SBTabHdr*>(ti.theta + F->rec_off),
                                     F->sbtab, it - ti.item0, ti.nitems, sh);
    __syncthreads();
  }
}

}  // namespace

int sigbkg_blocks_per_sm(bool mixed) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &nb, mixed ? k_sigbkg<true, true, false> : k_sigbkg<true, false, false>,
      sigbkg_threads(mixed), 0);
  cudaGetLastError();
  return nb > 0 ? nb : 1;
}

int sigbkg_threads(bool mixed) { return mixed ? sb_threads<true>() : sb_threads<false>(); }

cudaError_t launch_tick_sigbkg(bool mixed, const TickItem* items, int nfits, int total,
                               const WeidCoef& W, int sm_count, cudaStream_t st) {
  if (total <= 0) return cudaSuccess;
  const int grid = std::max(1, std::min(total, sm_count * (mixed ? sb_min_blocks<true>()
                                                                : sb_min_blocks<false>())));
  if (mixed) k_tick_sigbkg<true><<<grid, sb_threads<true>(), 0, st>>>(items, nfits, total, W);
  else k_tick_sigbkg<false><<<grid, sb_threads<false>(), 0, st>>>(items, nfits, total, W);
  return cudaGetLastError();
}

cudaError_t launch_sigbkg(const SigBkgDesc& D, const WeidCoef& W, const Program* prog,
                          const double* x, int64_t n,
                          const double* derived, double* partials, unsigned* counter,
                          double* result, double* out_logp, const int32_t* perm, bool grad,
                          bool mixed, int nblocks, const SBTabHdr* tab_hdr, const float4* tab,
                          cudaStream_t st) {
  if (nblocks < 1) nblocks = 1;
  const int NT = sigbkg_threads(mixed);
  auto go = [&](auto kern, double* lp, const int32_t* pm) {
    kern<<<nblocks, NT, 0, st>>>(D, W, prog, x, n, derived, partials, counter, result, lp, pm,
                                 tab_hdr, tab);
  };
  if (out_logp) {
    if (mixed) go(k_sigbkg<false, true, true>, out_logp, perm);
    else go(k_sigbkg<false, false, true>, out_logp, perm);
  } else if (mixed) {
    if (grad) go(k_sigbkg<true, true, false>, nullptr, nullptr);
    else go(k_sigbkg<false, true, false>, nullptr, nullptr);
  } else {
    if (grad) go(k_sigbkg<true, false, false>, nullptr, nullptr);
    else go(k_sigbkg<false, false, false>, nullptr, nullptr);
  }
  return cudaGetLastError();
}

// Layout of the table of w expansions for a Voigtian (mu, sigma, Gamma) over [lo, hi]:
// Re z = (x - mu) c1 with c1 = 1/(sigma sqrt2) and Im z = y = Gamma c1 / 2 as the leaf
// record forms them.  Core cells of width 2 x 0.96 of the FP64 plan's absolute limit
// (kSBLim64 or, y >= kSBLim64WY, kSBLim64W); for y >= 1e-6 logarithmic cells beyond
// |Re z| = 6 with half-widths 0.96 kSBLim64Rel |Re z|: the 4 % margin covers a rounded Re z
// or logarithm in the cell lookup.
void sbtab_layout(double mu, double sigma, double gamma, double lo, double hi, SBTabHdr& H) {
  H = SBTabHdr{};
  const double c1 = (1.0 / sigma) * (1.0 / kSqrt2);
  const double y = 0.5 * gamma * c1;
  if (!(sigma > 0.0) || !(gamma >= 0.0) || !std::isfinite(c1) || !std::isfinite(y) ||
      !(hi > lo))
    return;
  double zlo = (lo - mu) * c1, zhi = (hi - mu) * c1;
  const double pad = 1e-6 * (1.0 + std::max(std::fabs(zlo), std::fabs(zhi)));
  zlo -= pad;
  zhi += pad;
  const double h = 2.0 * 0.96 * (y >= kSBLim64WY ? (double)kSBLim64W : (double)kSBLim64);
  const bool wide = y >= 1e-6;
  const double zc = wide ? 6.0 : INFINITY;
  const double lr = std::log1p(2.0 * 0.96 * (double)kSBLim64Rel);
  const double a = std::max(-zc, zlo), b = std::min(zc, zhi);
  const double ncore = b > a ? std::ceil((b - a) / h) : 0.0;
  const double nneg = zlo < -zc ? std::ceil(std::log(-zlo / zc) / lr) : 0.0;
  const double npos = zhi > zc ? std::ceil(std::log(zhi / zc) / lr) : 0.0;
  const double nt = nneg + ncore + npos;
  if (!(nt >= 1.0 && nt <= (double)kSBTabCap)) return;
  H.ntab = (int32_t)nt;
  H.nneg = (int32_t)nneg;
  H.ncore = (int32_t)ncore;
  H.a = (float)a;
  H.ih = (float)(1.0 / h);
  H.h = (float)h;
  H.zc = (float)zc;
  H.izc = wide ? (float)(1.0 / zc) : 0.f;
  H.ilr = (float)(1.0 / lr);
  H.lr = (float)lr;
  H.mu = mu;
  H.c1 = c1;
  H.ic1 = sigma * kSqrt2;
  H.y = y;
}

// This unit's copy of the exp/log tables, once per device (that device current).
cudaError_t prepare_kernels_sigbkg() { return upload_df_tables(); }

}  // namespace gfi
