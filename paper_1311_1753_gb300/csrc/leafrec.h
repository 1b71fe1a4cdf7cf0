// leafrec.h -- leaf records of the analytically normalised leaves (exponential, Gaussian),
// shared by the device (k_1d.cu: every block's prologue, the normalisation kernel's last
// block) and the host (capi.cpp: the log-sum programs, whose records travel with theta).
// Record layout (kLeafRec doubles): [0] 1/N, [1] log N, [2..] d log N / d local parameter,
// [10..] the shape constants of the event arithmetic.
#pragma once

#include <cmath>

#include "gf_internal.h"

namespace gfi {

constexpr double kRecSqrt2 = 1.41421356237309504880;
constexpr double kRecSqrt2Pi = 2.50662827463100050242;

// L.kind L_EXP or L_GAUSS; rec zeroed by the caller.  raw: the unnormalised shape (N = 1).
__host__ __device__ inline void analytic_leaf_record(const LeafDesc& L, const double* th,
                                                     bool raw, double* rec) {
  const double lo = L.lo, hi = L.hi, D = hi - lo;
  double* c = rec + 10;
  if (L.kind == L_EXP) {
    // N = e^{a lo} expm1(a D)/a;  d log N/da = lo + D phi(aD),
    // phi(u) = 1/(1 - e^{-u}) - 1/u  (series 1/2 + u/12 - u^3/720 + u^5/30240 - u^7/1209600
    // for |u| < 0.1, Bernoulli numbers).
    const double a = th[L.par[0]];
    const double u = a * D;
    double logN, phi;
    if (a == 0.0) {
      logN = log(D);
      phi = 0.5;
    } else {
      logN = a * lo + log(expm1(u) / a);
      if (fabs(u) < 0.1) {
        const double u2 = u * u;
        phi = 0.5 + u * (1.0 / 12 + u2 * (-1.0 / 720 + u2 * (1.0 / 30240 - u2 / 1209600)));
      } else {
        phi = -1.0 / expm1(-u) - 1.0 / u;
      }
    }
    if (raw) logN = 0.0;
    rec[0] = exp(-logN);
    rec[1] = logN;
    rec[2] = raw ? 0.0 : lo + D * phi;
    c[0] = a;
    c[1] = -logN;
  } else {  // L_GAUSS
    const double mu = th[L.par[0]], s = th[L.par[1]];
    const double a = (lo - mu) / s, b = (hi - mu) / s;
    double diff;  // Phi(b) - Phi(a)
    if (a > 0.0) diff = 0.5 * (erfc(a / kRecSqrt2) - erfc(b / kRecSqrt2));
    else if (b < 0.0) diff = 0.5 * (erfc(-b / kRecSqrt2) - erfc(-a / kRecSqrt2));
    else diff = 0.5 * (erf(b / kRecSqrt2) - erf(a / kRecSqrt2));
    const double n = raw ? 1.0 : s * kRecSqrt2Pi * diff;
    const double ea = exp(-0.5 * a * a), eb = exp(-0.5 * b * b);
    rec[0] = 1.0 / n;
    rec[1] = log(n);
    rec[2] = raw ? 0.0 : (ea - eb) / n;
    rec[3] = raw ? 0.0 : (a * ea - b * eb) / n + 1.0 / s;
    c[0] = mu;
    c[1] = 1.0 / s;
    c[2] = -rec[1];
  }
}

}  // namespace gfi
