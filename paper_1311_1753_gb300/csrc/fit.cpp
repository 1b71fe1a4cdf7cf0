// fit.cpp -- the quasi-Newton minimiser behind gf_fit (Sec. 2 of the paper: FitManager
// defines each parameter to MINUIT and runs Migrad; the paper notes any search
// algorithm may take its place).
//
// BFGS on MINUIT's internal coordinates: a parameter with limits lo < hi is
//   ext = lo + (hi - lo) (sin(u) + 1)/2,
// unbounded ones are used as they are.  The step is chosen by a line search meeting the
// strong Wolfe conditions (bracketing, then cubic-interpolation zoom).  Convergence:
// EDM = g^T V g / 2 < tol with V the inverse-Hessian estimate (MINUIT's criterion).
// Parabolic errors: Hessian in external coordinates by central differences of the
// analytic gradient at the minimum, covariance = 2 up H^-1.
#include "fit.h"

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/gf.h"
#include "ctx.h"

namespace gfi {

namespace {

struct Bounds {
  std::vector<double> lo, hi;
  bool b(size_t k) const { return hi[k] > lo[k]; }
  double ext(size_t k, double u) const {
    return b(k) ? lo[k] + (hi[k] - lo[k]) * (std::sin(u) + 1.0) * 0.5 : u;
  }
  double der(size_t k, double u) const { return b(k) ? (hi[k] - lo[k]) * std::cos(u) * 0.5 : 1.0; }
  double inv(size_t k, double x) const {
    if (!b(k)) return x;
    double r = 2.0 * (x - lo[k]) / (hi[k] - lo[k]) - 1.0;
    r = std::max(-1.0, std::min(1.0, r));
    return std::asin(r);
  }
};

// Minimiser of the cubic through (a, fa, da), (b, fb, db), clamped into the bracket.
double cubic_min(double a, double fa, double da, double b, double fb, double db) {
  const double d1 = da + db - 3.0 * (fa - fb) / (a - b);
  const double s = d1 * d1 - da * db;
  if (s < 0) return 0.5 * (a + b);
  double d2 = std::sqrt(s);
  if (b < a) d2 = -d2;
  const double t = b - (b - a) * (db + d2 - d1) / (db - da + 2.0 * d2);
  const double lo = std::min(a, b), hi = std::max(a, b);
  const double w = hi - lo;
  if (!std::isfinite(t) || t < lo + 0.1 * w || t > hi - 0.1 * w) return 0.5 * (a + b);
  return t;
}

}  // namespace

MinResult minimise(const FGFun& fg, const std::vector<double>& x0, const std::vector<double>& step,
                   const std::vector<double>& lo, const std::vector<double>& hi,
                   const MinOpts& opt) {
  const size_t n = x0.size();
  MinResult res;
  Bounds B{lo, hi};
  std::vector<double> u(n), x(n), g(n), gext(n);
  for (size_t k = 0; k < n; ++k) u[k] = B.inv(k, x0[k]);
  int calls = 0;
  int fail = 0;
  // f and internal gradient at internal point v
  auto eval = [&](const std::vector<double>& v, double& f, std::vector<double>& gi) -> int {
    std::vector<double> xe(n);
    for (size_t k = 0; k < n; ++k) xe[k] = B.ext(k, v[k]);
    std::vector<double> ge(n, 0.0);
    ++calls;
    int rc = fg(xe, f, ge);
    if (rc != GF_OK && rc != GF_ENONFINITE) return rc;
    if (rc == GF_ENONFINITE || !std::isfinite(f)) {
      f = INFINITY;
      return GF_ENONFINITE;
    }
    gi.resize(n);
    for (size_t k = 0; k < n; ++k) gi[k] = ge[k] * B.der(k, v[k]);
    return GF_OK;
  };
  double f;
  int rc = eval(u, f, g);
  if (rc != GF_OK) {
    res.status = rc;
    res.calls = calls;
    return res;
  }
  // V0 = diag(step_int^2), or the caller's estimate
  std::vector<double> V(n * n, 0.0), sint(n);
  for (size_t k = 0; k < n; ++k) {
    const double d = std::max(std::fabs(B.der(k, u[k])), 1e-300);
    sint[k] = step[k] / d;
    V[k * n + k] = sint[k] * sint[k];
  }
  const bool given_V = opt.V0 && opt.V0->size() == n * n;
  if (given_V) V = *opt.V0;
  auto edm_of = [&](const std::vector<double>& gg) {
    double e = 0.0;
    for (size_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (size_t j = 0; j < n; ++j) s += V[i * n + j] * gg[j];
      e += gg[i] * s;
    }
    return 0.5 * e;
  };
  double edm = edm_of(g);
  std::vector<double> p(n), un(n), gn(n), s(n), y(n), Vy(n);
  int it = 0;
  bool converged = edm < opt.tol;
  for (; !converged && it < 10000 && calls < opt.max_calls; ++it) {
    // direction p = -V g
    double d0 = 0.0;
    for (size_t i = 0; i < n; ++i) {
      double a = 0.0;
      for (size_t j = 0; j < n; ++j) a += V[i * n + j] * g[j];
      p[i] = -a;
      d0 += g[i] * p[i];
    }
    if (!(d0 < 0)) {  // lost positive definiteness: restart from the diagonal
      std::fill(V.begin(), V.end(), 0.0);
      for (size_t k = 0; k < n; ++k) V[k * n + k] = sint[k] * sint[k];
      for (size_t i = 0; i < n; ++i) p[i] = -V[i * n + i] * g[i];
      d0 = 0.0;
      for (size_t i = 0; i < n; ++i) d0 += g[i] * p[i];
      if (!(d0 < 0)) break;
    }
    // strong-Wolfe line search along p
    const double c1 = 1e-4, c2 = 0.9;
    const double fn = opt.f_noise_rel * std::fabs(f);  // differences below the noise
                                                        // count as no change
    auto phi = [&](double a, double& fa, double& da, std::vector<double>& ga) -> int {
      for (size_t i = 0; i < n; ++i) un[i] = u[i] + a * p[i];
      int r = eval(un, fa, ga);
      da = 0.0;
      if (r == GF_OK)
        for (size_t i = 0; i < n; ++i) da += ga[i] * p[i];
      return r;
    };
    double a_prev = 0.0, f_prev = f, d_prev = d0;
    double a = 1.0, fa = 0, da = 0;
    double a_ok = -1.0, f_ok = 0;
    std::vector<double> g_ok(n), ga(n);
    bool hard = false;
    for (int ls = 0; ls < 30 && calls < opt.max_calls; ++ls) {
      int r = phi(a, fa, da, ga);
      if (r != GF_OK && r != GF_ENONFINITE) { hard = true; rc = r; break; }
      if (r == GF_ENONFINITE) { a = 0.5 * (a_prev + a); continue; }
      if (fa > f + c1 * a * d0 + fn || (ls > 0 && fa >= f_prev + fn)) {
        // zoom in [a_prev, a]
        double alo = a_prev, flo = f_prev, dlo = d_prev, ahi = a, fhi = fa, dhi = da;
        for (int z = 0; z < 30 && calls < opt.max_calls; ++z) {
          const double at = cubic_min(alo, flo, dlo, ahi, fhi, dhi);
          double ft, dt;
          int rz = phi(at, ft, dt, ga);
          if (rz != GF_OK && rz != GF_ENONFINITE) { hard = true; rc = rz; break; }
          if (rz == GF_ENONFINITE || ft > f + c1 * at * d0 + fn || ft >= flo + fn) {
            ahi = at; fhi = (rz == GF_OK) ? ft : INFINITY; dhi = (rz == GF_OK) ? dt : 0.0;
            if (rz != GF_OK) { fhi = flo + 1.0; dhi = -dlo; }
          } else {
            if (std::fabs(dt) <= -c2 * d0) { a_ok = at; f_ok = ft; g_ok = ga; break; }
            if (dt * (ahi - alo) >= 0) { ahi = alo; fhi = flo; dhi = dlo; }
            alo = at; flo = ft; dlo = dt;
            a_ok = at; f_ok = ft; g_ok = ga;  // best so far satisfies sufficient decrease
          }
          if (std::fabs(ahi - alo) < 1e-14 * std::max(1.0, std::fabs(alo))) break;
        }
        break;
      }
      if (std::fabs(da) <= -c2 * d0) { a_ok = a; f_ok = fa; g_ok = ga; break; }
      if (da >= 0) {
        double alo = a, flo = fa, dlo = da, ahi = a_prev, fhi = f_prev, dhi = d_prev;
        a_ok = a; f_ok = fa; g_ok = ga;
        for (int z = 0; z < 30 && calls < opt.max_calls; ++z) {
          const double at = cubic_min(alo, flo, dlo, ahi, fhi, dhi);
          double ft, dt;
          int rz = phi(at, ft, dt, ga);
          if (rz != GF_OK && rz != GF_ENONFINITE) { hard = true; rc = rz; break; }
          if (rz == GF_ENONFINITE || ft > f + c1 * at * d0 + fn || ft >= flo + fn) {
            ahi = at; fhi = (rz == GF_OK) ? ft : flo + 1.0; dhi = (rz == GF_OK) ? dt : -dlo;
          } else {
            if (std::fabs(dt) <= -c2 * d0) { a_ok = at; f_ok = ft; g_ok = ga; break; }
            if (dt * (ahi - alo) >= 0) { ahi = alo; fhi = flo; dhi = dlo; }
            alo = at; flo = ft; dlo = dt;
            a_ok = at; f_ok = ft; g_ok = ga;
          }
          if (std::fabs(ahi - alo) < 1e-14 * std::max(1.0, std::fabs(alo))) break;
        }
        break;
      }
      a_prev = a; f_prev = fa; d_prev = da;
      a_ok = a; f_ok = fa; g_ok = ga;
      a *= 2.0;
    }
    if (hard) break;
    if (a_ok <= 0 || !(f_ok < f + fn)) {
      if (++fail >= 2) break;
      std::fill(V.begin(), V.end(), 0.0);
      for (size_t k = 0; k < n; ++k) V[k * n + k] = sint[k] * sint[k];
      continue;
    }
    fail = 0;
    for (size_t i = 0; i < n; ++i) {
      s[i] = a_ok * p[i];
      y[i] = g_ok[i] - g[i];
    }
    double sy = 0.0, yy = 0.0;
    for (size_t i = 0; i < n; ++i) { sy += s[i] * y[i]; yy += y[i] * y[i]; }
    if (it == 0 && sy > 0 && !given_V) {
      // rescale the initial estimate (Nocedal & Wright, eq. 6.20)
      std::fill(V.begin(), V.end(), 0.0);
      for (size_t k = 0; k < n; ++k) V[k * n + k] = sy / yy;
    }
    if (sy > 1e-300) {
      // V <- (I - rho s y^T) V (I - rho y s^T) + rho s s^T
      const double rho = 1.0 / sy;
      for (size_t i = 0; i < n; ++i) {
        double a2 = 0.0;
        for (size_t j = 0; j < n; ++j) a2 += V[i * n + j] * y[j];
        Vy[i] = a2;
      }
      double yVy = 0.0;
      for (size_t i = 0; i < n; ++i) yVy += y[i] * Vy[i];
      for (size_t i = 0; i < n; ++i)
        for (size_t j = 0; j < n; ++j)
          V[i * n + j] += -rho * (s[i] * Vy[j] + Vy[i] * s[j]) + (rho * rho * yVy + rho) * s[i] * s[j];
    }
    for (size_t i = 0; i < n; ++i) u[i] += s[i];
    f = f_ok;
    g = g_ok;
    edm = edm_of(g);
    converged = edm < opt.tol;
  }
  res.iters = it;
  res.fval = f;
  res.edm = edm;
  res.converged = converged;
  res.x.resize(n);
  for (size_t k = 0; k < n; ++k) res.x[k] = B.ext(k, u[k]);
  if (rc != GF_OK && rc != GF_ENONFINITE) {
    res.status = rc;
    res.calls = calls;
    return res;
  }
  res.status = converged ? GF_OK : GF_ENOCONV;
  res.V = V;
  res.err.assign(n, 0.0);
  res.cov.assign(n * n, 0.0);
  if (opt.hesse && n > 0) hesse(fg, res.x, V, lo, hi, opt.up, res.err, res.cov, &calls);
  res.calls = calls;
  return res;
}

bool hesse(const FGFun& fg, const std::vector<double>& x, const std::vector<double>& V,
           const std::vector<double>& lo, const std::vector<double>& hi, double up,
           std::vector<double>& err, std::vector<double>& cov, int* calls) {
  const size_t n = x.size();
  Bounds B{lo, hi};
  std::vector<double> H(n * n), gp(n), gm(n), xp(n);
  for (size_t k = 0; k < n; ++k) {
    // step: 1% of the error estimate from V mapped to external units
    const double u = B.inv(k, x[k]);
    const double sig = std::sqrt(std::fabs(V[k * n + k])) * std::fabs(B.der(k, u));
    double h = sig > 0 ? 1e-2 * sig : 1e-6 * std::max(1.0, std::fabs(x[k]));
    if (B.b(k)) h = std::min(h, 0.25 * std::min(x[k] - lo[k], hi[k] - x[k]) + 1e-300);
    xp = x;
    xp[k] += h;
    double fp, fm;
    ++*calls;
    if (fg(xp, fp, gp) != GF_OK) return false;
    xp[k] = x[k] - h;
    ++*calls;
    if (fg(xp, fm, gm) != GF_OK) return false;
    for (size_t i = 0; i < n; ++i) H[i * n + k] = (gp[i] - gm[i]) / (2.0 * h);
  }
  for (size_t i = 0; i < n; ++i)
    for (size_t j = i + 1; j < n; ++j) {
      const double m = 0.5 * (H[i * n + j] + H[j * n + i]);
      H[i * n + j] = H[j * n + i] = m;
    }
  // invert by Gauss-Jordan with partial pivoting
  std::vector<double> A = H, I(n * n, 0.0);
  for (size_t k = 0; k < n; ++k) I[k * n + k] = 1.0;
  for (size_t c = 0; c < n; ++c) {
    size_t piv = c;
    for (size_t r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    if (piv != c)
      for (size_t j = 0; j < n; ++j) {
        std::swap(A[c * n + j], A[piv * n + j]);
        std::swap(I[c * n + j], I[piv * n + j]);
      }
    const double d = 1.0 / A[c * n + c];
    for (size_t j = 0; j < n; ++j) {
      A[c * n + j] *= d;
      I[c * n + j] *= d;
    }
    for (size_t r = 0; r < n; ++r)
      if (r != c) {
        const double m = A[r * n + c];
        if (m != 0.0)
          for (size_t j = 0; j < n; ++j) {
            A[r * n + j] -= m * A[c * n + j];
            I[r * n + j] -= m * I[c * n + j];
          }
      }
  }
  for (size_t k = 0; k < n * n; ++k) cov[k] = 2.0 * up * I[k];
  for (size_t k = 0; k < n; ++k) err[k] = std::sqrt(std::fabs(cov[k * n + k]));
  return true;
}

MinResult minimise_refined(const FGFun* fg_fast, const FGFun& fg_exact,
                           const std::vector<double>& x0, const std::vector<double>& step,
                           const std::vector<double>& lo, const std::vector<double>& hi,
                           const MinOpts& opt) {
  if (!fg_fast) return minimise(fg_exact, x0, step, lo, hi, opt);
  MinOpts o1 = opt;
  o1.tol = std::max(opt.tol, 1.0);
  o1.hesse = false;
  o1.f_noise_rel = opt.f_noise_rel_fast;
  MinResult r1 = minimise(*fg_fast, x0, step, lo, hi, o1);
  if (r1.x.empty() || (r1.status != GF_OK && r1.status != GF_ENOCONV)) return r1;
  MinOpts o2 = opt;
  o2.hesse = false;
  // the FP64-accurate sums' own rounding (pair accumulators: ~1e-15 of |f| for millions of
  // events): below it a line search cannot tell a step's decrease from noise
  o2.f_noise_rel = opt.f_noise_rel_exact;
  o2.max_calls = std::max(1, opt.max_calls - r1.calls);
  // curvature for the FP64 stage: the FP32 Hessian at the hand-over point, mapped to
  // internal coordinates (V = D^-1 H_ext^-1 D^-1, D = dext/du); BFGS's own estimate
  // after a few FP32 iterations is too rough for 30 parameters
  const size_t n = r1.x.size();
  std::vector<double> e1(n), c1(n * n), V0 = r1.V;
  int hc1 = 0;
  if (n > 0 && hesse(*fg_fast, r1.x, r1.V, lo, hi, opt.up, e1, c1, &hc1)) {
    Bounds B{lo, hi};
    std::vector<double> d(n);
    for (size_t k = 0; k < n; ++k) d[k] = B.der(k, B.inv(k, r1.x[k]));
    bool ok = true;
    for (size_t i = 0; i < n && ok; ++i)
      for (size_t j = 0; j < n; ++j) {
        const double v = c1[i * n + j] / (2.0 * opt.up) / (d[i] * d[j]);
        if (!std::isfinite(v)) ok = false;
        V0[i * n + j] = v;
      }
    if (!ok) V0 = r1.V;
  }
  r1.calls += hc1;
  o2.V0 = &V0;
  MinResult r2 = minimise(fg_exact, r1.x, step, lo, hi, o2);
  r2.calls_fast = r1.calls;
  r2.calls += r1.calls;
  r2.iters += r1.iters;
  if (r2.x.empty()) return r2;
  r2.err.assign(r2.x.size(), 0.0);
  r2.cov.assign(r2.x.size() * r2.x.size(), 0.0);
  if (opt.hesse && !r2.x.empty()) {
    int hc = 0;
    hesse(*fg_fast, r2.x, r2.V, lo, hi, opt.up, r2.err, r2.cov, &hc);
    r2.calls += hc;
    r2.calls_fast += hc;
  }
  return r2;
}

}  // namespace gfi

using namespace gfi;

extern "C" int gf_fit(gf_ctx* ctx, const gf_fit_opts* opts, gf_fit_result* res) {
  if (!ctx || !res || !res->theta) return GF_EINVAL;
  int rc = ensure_compiled(ctx);
  if (rc) return rc;
  MinOpts mo;
  mo.up = ctx->metric == GF_METRIC_CHISQ ? 1.0 : 0.5;  // chi-squared: Delta chi2 = 1
  bool use_grad = true;
  if (opts) {
    if (opts->tol > 0) mo.tol = opts->tol;
    if (opts->max_calls > 0) mo.max_calls = opts->max_calls;
    if (opts->up > 0) mo.up = opts->up;
    mo.hesse = opts->hesse != 0;
    use_grad = opts->use_grad != 0;
  }
  const size_t n = ctx->free_ids.size();
  std::vector<double> x0(n), step(n), lo(n), hi(n);
  for (size_t k = 0; k < n; ++k) {
    const ParDef& p = ctx->pars[ctx->free_ids[k]];
    x0[k] = p.value;
    step[k] = p.step;
    lo[k] = p.lo;
    hi[k] = p.hi;
  }
  auto make_fg = [&](bool fp64) -> FGFun {
    return [&, fp64](const std::vector<double>& x, double& f, std::vector<double>& g) -> int {
    if (use_grad) return evaluate(ctx, x.data(), &f, g.data(), fp64);
    int r = evaluate(ctx, x.data(), &f, nullptr, fp64);
    if (r) return r;
    // central differences of the NLL, 2 n extra evaluations
    std::vector<double> xp = x;
    for (size_t k = 0; k < n; ++k) {
      const double h = 1e-3 * step[k];
      double fp, fm;
      xp[k] = x[k] + h;
      r = evaluate(ctx, xp.data(), &fp, nullptr, fp64);
      if (r) return r;
      xp[k] = x[k] - h;
      r = evaluate(ctx, xp.data(), &fm, nullptr, fp64);
      if (r) return r;
      xp[k] = x[k];
      g[k] = (fp - fm) / (2 * h);
    }
    return GF_OK;
    };
  };
  // mixed contexts: FP32 BFGS, then an FP64 polish from the FP32 inverse Hessian
  // (only Dalitz models and the signal + background form have an FP32 plan; other 1D
  // programs evaluate FP64-accurate in every context: nothing to refine)
  const bool refine = ctx->precision == GF_MIXED && (ctx->is_dalitz || ctx->use_sb) &&
                      (!opts || opts->refine != 0);
  FGFun fg_fast = make_fg(false), fg_exact = make_fg(ctx->precision == GF_MIXED);
  MinResult m = refine ? minimise_refined(&fg_fast, fg_exact, x0, step, lo, hi, mo)
                       : minimise(fg_fast, x0, step, lo, hi, mo);
  res->nll = m.fval;
  res->edm = m.edm;
  res->n_calls = m.calls;
  res->n_iter = m.iters;
  res->n_calls_fast = m.calls_fast;
  res->status = m.status;
  if (!m.x.empty()) {
    for (size_t k = 0; k < n; ++k) {
      res->theta[k] = m.x[k];
      ctx->pars[ctx->free_ids[k]].value = m.x[k];
      if (res->err) res->err[k] = m.err[k];
    }
    if (res->cov)
      for (size_t k = 0; k < n * n; ++k) res->cov[k] = m.cov[k];
  }
  return m.status;
}
