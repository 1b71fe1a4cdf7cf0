// devutil.cuh -- device helpers of the sm_103a kernels: deterministic block
// reductions, the last-block completion pattern, and the Faddeeva function.
#pragma once
#include <cuda_runtime.h>
#include "df64.cuh"
#include "gf_internal.h"

namespace gfi {

constexpr double kInvSqrtPi = 0.56418958354775628695;  // 1/sqrt(pi)
constexpr double kTwoInvSqrtPi = 1.12837916709551257390;
constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double kInvSqrt2 = 0.70710678118654752440;
constexpr double kSqrt2Pi = 2.50662827463100050242;
constexpr double kInvSqrt2Pi = 0.39894228040143267794;  // 1/sqrt(2 pi)

// ---- compensated accumulation ------------------------------------------------------
// FP64: plain sum (a thread adds O(100) terms).  FP32: Kahan pair, converted to FP64
// when the thread hands its sum to the block reduction.
template <typename T>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double get() const { return s; }
};
template <>
struct Acc<DF> {
  DF s = DF(0.f);
  __device__ __forceinline__ void add(DF v) { s += v; }
  __device__ __forceinline__ double get() const { return s.to_double(); }
  __device__ __forceinline__ F2 pair() const { return s; }
};
template <>
struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double get() const { return (double)s - (double)c; }
  __device__ __forceinline__ F2 pair() const { return two_sum(s, -c); }
};

// ---- warp / block reductions in a fixed order (bitwise reproducible) -------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Reduce one value over the block; result valid in thread 0.  `red` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) r += red[w];
  return r;
}

// Neumaier pair for the cross-block pass.
struct Neu {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double v) {
    double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
  }
  __device__ __forceinline__ double get() const { return s + c; }
};

// Block-wide fixed-order sum of partials[b * stride + k] over b < nblk, for each
// k < m; writes out[k].  Called by every thread of one block.

// Sum m per-thread values (pairs, from val(k)) over the block in a fixed order and write
// the block's sums to out[0 .. m-1] (global memory): each warp folds its 32 lanes with
// pair shuffles (lane order fixed), lane 0 stores the warp's m sums as pairs in
// red[warp * m + k], one barrier, then thread k adds the warps' k-th sums as pairs and
// converts the total to FP64 once.  Every step stays on the FP32 pipe until that one
// conversion per value (an FP64 instruction occupies an SM sub-partition for many cycles
// on this part, so per-warp conversions of every value were the slow part).
// red: (blockDim / 32) * m doubles (each slot holds one pair).
// M >= 0: the count m known at compile time (the loop unrolls, val's index is a constant,
// so a caller's per-thread array stays in registers).
template <int M = -1, class Val>
__device__ __forceinline__ void block_sum_pairs(Val val, int m, double* red, double* out,
                                                int ostride = 1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (M >= 0) {
    m = M;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      F2 v = val(k);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const F2 u = {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
        v = df_add(v, u);
      }
      if (lane == 0) reinterpret_cast<F2*>(red)[warp * m + k] = v;
    }
  } else {
    // values four at a time, their shuffle trees interleaved (the same tree per value)
    for (int k0 = 0; k0 < m; k0 += 4) {
      F2 v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = k0 + j < m ? val(k0 + j) : F2{0.f, 0.f};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const F2 u = {__shfl_down_sync(0xffffffffu, v[j].hi, o),
                        __shfl_down_sync(0xffffffffu, v[j].lo, o)};
          v[j] = df_add(v[j], u);
        }
      }
      if (lane == 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (k0 + j < m) reinterpret_cast<F2*>(red)[warp * m + k0 + j] = v[j];
      }
    }
  }
  __syncthreads();
  const F2* rp = reinterpret_cast<const F2*>(red);
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    F2 r = rp[k];
    for (int w = 1; w < nw; ++w) r = df_add(r, rp[w * m + k]);
    out[(size_t)k * ostride] = df_to(r);
  }
}

// Cross-block sums by the last block: out[k] = sum over b < nblk of
// partials[b stride + k kstride], k < m, in a fixed order.  Warp w takes k = w, w + nwarps,
// ...; its lanes stride over the blocks with all their loads in flight (kPer per lane and
// pass), summing as pairs in two interleaved chains (partials enter by the bit split: no
// FP64 conversions; the padding zeros add exactly), then a fixed shuffle tree.  The
// value-major layout (stride 1, kstride >= nblk) makes each warp load one contiguous run
// of 256 bytes; the block-major one (kstride 1) touches a line per lane.  Called by every
// thread of one block; ends with a barrier.
template <int kPer = 16>
__device__ inline void reduce_partials(const double* partials, int nblk, int stride, int m,
                                       double* out, int kstride = 1) {
  static_assert(kPer % 2 == 0, "two chains");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = warp; k < m; k += nw) {
    const double* p = partials + (size_t)k * kstride;
    F2 a = {0.f, 0.f}, a2 = {0.f, 0.f};
    for (int b0 = 0; b0 < nblk; b0 += 32 * kPer) {
      double v[kPer];
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int b = b0 + lane + 32 * j;
        v[j] = b < nblk ? __ldcg(p + (size_t)b * stride) : 0.0;
      }
      // only the loaded values: the padding is skipped, not split (df_split takes a
      // zero down its out-of-line conversion path)
#pragma unroll
      for (int j = 0; j < kPer; j += 2) {
        if (b0 + lane + 32 * j < nblk) a = df_add(a, df_split(v[j]));
        if (b0 + lane + 32 * (j + 1) < nblk) a2 = df_add(a2, df_split(v[j + 1]));
      }
    }
    a = df_add(a, a2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const F2 u = {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
      a = df_add(a, u);
    }
    if (lane == 0) out[k] = df_to(a);
  }
  __syncthreads();
}

// Padded block-major partials: value k of block b at partials[b ps + k] with ps the
// smallest multiple of 16 doubles >= m, so that every block writes its own 128-byte lines
// (in the value-major layout 16 blocks' 8-byte stores share a line).
__host__ __device__ constexpr int partial_stride(int m) { return (m + 15) / 16 * 16; }

// Their cross-block sums by the last block: thread t sums the elements t, t + T, t + 2T, ...
// of the flat array (value t mod ps for T a multiple of ps; consecutive threads load
// consecutive doubles, kB loads in flight) as pairs, then thread k < m adds the T/ps sums of
// value k in order and converts once.  Fixed order (bitwise reproducible).  scratch: T
// pairs (shared memory); out: m doubles.  Called by every thread of one block; ends with a
// barrier.
template <int kB = 8>
__device__ inline void reduce_partials_bm(const double* partials, int nblk, int m, double* out,
                                          F2* scratch) {
  const int T = blockDim.x, t = threadIdx.x, ps = partial_stride(m);
  if (T % ps != 0) {  // a warp per value over the same layout
    reduce_partials(partials, nblk, ps, m, out, 1);
    return;
  }
  const int total = nblk * ps;
  F2 a = {0.f, 0.f}, a2 = {0.f, 0.f};
  if (t % ps < m) {
    for (int f0 = t; f0 < total; f0 += kB * T) {
      double v[kB];
#pragma unroll
      for (int j = 0; j < kB; ++j) {
        const int f = f0 + j * T;
        v[j] = f < total ? __ldcg(partials + f) : 0.0;
      }
#pragma unroll
      for (int j = 0; j < kB; j += 2) {  // only the loaded values (df_split's zero path is a call)
        if (f0 + j * T < total) a = df_add(a, df_split(v[j]));
        if (f0 + (j + 1) * T < total) a2 = df_add(a2, df_split(v[j + 1]));
      }
    }
  }
  scratch[t] = df_add(a, a2);
  __syncthreads();
  if (t < m) {
    F2 r = scratch[t];
    for (int j = t + ps; j < T; j += ps) r = df_add(r, scratch[j]);
    out[t] = df_to(r);
  }
  __syncthreads();
}

// Last-block pattern: every block publishes its partial, then bumps a counter; the
// block that takes the last ticket sees every partial and finishes the reduction.
// The counter is reset by that block, so the next launch starts from zero.
__device__ __forceinline__ bool arrive_last_of(unsigned* counter, unsigned expected,
                                               int* flag_smem) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    *flag_smem = (t == expected - 1) ? 1 : 0;
  }
  __syncthreads();
  const bool last = *flag_smem != 0;
  if (last) __threadfence();
  return last;
}
__device__ __forceinline__ bool arrive_last(unsigned* counter, int* flag_smem) {
  return arrive_last_of(counter, gridDim.x * gridDim.y, flag_smem);
}

// ---- Faddeeva function w(z) = exp(-z^2) erfc(-iz), Im z >= 0 ---------------------------
// Weideman (1994), "Computation of the complex error function", SIAM J. Numer. Anal.
// 31, 1497: expand (L^2 + t^2) e^{-t^2} in powers of Z(t) = (L + it)/(L - it), which maps
// the real line onto the unit circle; integrating the Cauchy representation term by
// term (residues at t = z and, for the constant term, t = iL) gives
//   w(z) = 1/(sqrt(pi) (L - iz)) + 2/(L - iz)^2 sum_{n=1}^{N} a_n Z^{n-1},
//   Z = (L + iz)/(L - iz),  L = 2^{-1/4} sqrt(N).
// The a_n are Fourier coefficients computed on the host (WeidCoef).  N = 40 gives |w|
// to ~2e-14 relative over the Voigtian's range of z.  FP64-accurate version on the FP32
// pipe: every step in double-float, except the high-order terms n >= kWeidSplit, whose
// coefficients are below 4e-9 (a_1 = 2.9): their partial sum is formed in plain float,
// which changes w by < 1e-18 absolute (3e-14 relative to Re w at |Re z| = 37).
constexpr int kWeidSplit = 24;
__device__ __forceinline__ void faddeeva_f2(F2 X, F2 Y, const WeidCoef& W, F2& WR, F2& WI) {
  const F2 L = {W.Lhi, W.Llo};
  const F2 dr = df_add(L, Y);                                        // L - iz = dr - i x
  const F2 x2 = df_mul(X, X);
  const F2 inv = df_rcp(df_add(df_mul(dr, dr), x2));                 // 1/|L - iz|^2
  const F2 zr = df_mul(df_sub(df_mul(df_sub(L, Y), dr), x2), inv);   // Re Z
  const F2 zi = df_mul(df_mul_f(df_mul(L, X), 2.f), inv);            // Im Z
  // tail n = N .. kWeidSplit in float
  float fr = W.ahi[kWeidN], fi = 0.f;
#pragma unroll
  for (int n = kWeidN - 1; n >= kWeidSplit; --n) {
    const float t = __fmaf_rn(fr, zr.hi, __fmaf_rn(-fi, zi.hi, W.ahi[n]));
    fi = __fmaf_rn(fr, zi.hi, __fmul_rn(fi, zr.hi));
    fr = t;
  }
  F2 pr = {fr, 0.f}, pi = {fi, 0.f};
  // rolled: one copy of the step stays in the instruction cache (W sits in the constant
  // bank, a __grid_constant__ kernel parameter, so W.ahi[n] is an indexed constant load)
#pragma unroll 1
  for (int n = kWeidSplit - 1; n >= 1; --n) {
    // real: pr zr - pi zi + a_n ; imag: pr zi + pi zr
    const F2 t1 = df_mul_raw(pr, zr), t2 = df_mul_raw(pi, zi);
    const F2 s1 = two_sum(t1.hi, -t2.hi);
    const F2 s2 = two_sum(s1.hi, W.ahi[n]);
    const float er =
        __fadd_rn(__fadd_rn(__fadd_rn(s1.lo, s2.lo), __fsub_rn(t1.lo, t2.lo)), W.alo[n]);
    const F2 t3 = df_mul_raw(pr, zi), t4 = df_mul_raw(pi, zr);
    const F2 s3 = two_sum(t3.hi, t4.hi);
    const float ei = __fadd_rn(s3.lo, __fadd_rn(t3.lo, t4.lo));
    pr = fast_two_sum(s2.hi, er);
    pi = fast_two_sum(s3.hi, ei);
  }
  const F2 ir = df_mul(dr, inv), ii = df_mul(X, inv);                // 1/(L - iz)
  const F2 qr = df_sub(df_mul(ir, ir), df_mul(ii, ii));              // 1/(L - iz)^2
  const F2 qi = df_mul_f(df_mul(ir, ii), 2.f);
  constexpr DFC c(kInvSqrtPi);
  WR = df_add(df_mul(c, ir), df_mul_f(df_sub(df_mul(pr, qr), df_mul(pi, qi)), 2.f));
  WI = df_add(df_mul(c, ii), df_mul_f(df_add(df_mul(pr, qi), df_mul(pi, qr)), 2.f));
}
// erfcx(y) = w(i y) for real y >= 0 by the same series: with z = i y, L - iz = L + y and
// Z = (L - y)/(L + y) are real, so erfcx(y) = (1/sqrt(pi) + 2 P(Z)/(L + y))/(L + y) with
// P(Z) = sum_n a_n Z^{n-1}; real pair arithmetic, the high-order terms in float as above.
// FP64 in and out.
__device__ __forceinline__ double erfcx_df(double y, const WeidCoef& W) {
  const F2 L = {W.Lhi, W.Llo}, Y = df_from(y);
  const F2 ir = df_rcp(df_add(L, Y));                                // 1/(L + y)
  const F2 z = df_mul(df_sub(L, Y), ir);
  float f = W.ahi[kWeidN];
#pragma unroll
  for (int n = kWeidN - 1; n >= kWeidSplit; --n) f = __fmaf_rn(f, z.hi, W.ahi[n]);
  F2 p = {f, 0.f};
#pragma unroll 1
  for (int n = kWeidSplit - 1; n >= 1; --n) p = df_add(df_mul(p, z), F2{W.ahi[n], W.alo[n]});
  constexpr DFC c(kInvSqrtPi);
  return df_to(df_mul(df_add(c, df_mul_f(df_mul(p, ir), 2.f)), ir));
}
// FP64 in and out (the normalisation grid)
__device__ __forceinline__ void faddeeva_df(double x, double y, const WeidCoef& W, double& wr,
                                            double& wi) {
  F2 WR, WI;
  faddeeva_f2(df_from(x), df_from(y), W, WR, WI);
  wr = df_to(WR);
  wi = df_to(WI);
}

}  // namespace gfi
