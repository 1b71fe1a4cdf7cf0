// fit.h -- host quasi-Newton minimiser shared by gf_fit and the fit server.
#pragma once
#include <functional>
#include <vector>

namespace gfi {

struct MinOpts {
  double tol = 1e-6;   // EDM tolerance
  int max_calls = 5000;
  double up = 0.5;
  bool hesse = true;
  const std::vector<double>* V0 = nullptr;  // starting inverse Hessian (internal coords)
  double f_noise_rel = 0.0;       // noise of f relative to |f|: smaller differences count as
                                  // no change in the line search
  double f_noise_rel_fast = 3e-8; // the same for fg_fast of minimise_refined (FP32 sums)
  double f_noise_rel_exact = 2e-15;  // ... and for its FP64-accurate stage
};

struct MinResult {
  std::vector<double> x, err, cov;
  std::vector<double> V;  // final inverse-Hessian estimate (internal coordinates)
  double fval = 0.0, edm = 0.0;
  int calls = 0, iters = 0;
  int calls_fast = 0;  // minimise_refined: evaluations made on fg_fast
  bool converged = false;
  int status = 0;  // GF_OK / GF_ENOCONV / evaluation error code
};

// f(x, g) -> status; x in external units; g (same length) filled with df/dx.
using FGFun = std::function<int(const std::vector<double>&, double&, std::vector<double>&)>;

MinResult minimise(const FGFun& fg, const std::vector<double>& x0, const std::vector<double>& step,
                   const std::vector<double>& lo, const std::vector<double>& hi,
                   const MinOpts& opt);

// Parabolic errors at x: Hessian of f in external coordinates by central differences of
// the gradient (steps from the internal inverse-Hessian estimate V), cov = 2 up H^-1.
bool hesse(const FGFun& fg, const std::vector<double>& x, const std::vector<double>& V,
           const std::vector<double>& lo, const std::vector<double>& hi, double up,
           std::vector<double>& err, std::vector<double>& cov, int* calls);

// A fit in two precisions: BFGS on fg_fast (FP32 amplitudes) to EDM < max(tol, 1), or
// until its noise stops the line search, then BFGS on fg_exact (FP64) from that point and
// inverse-Hessian estimate to EDM < tol; errors from the Hessian of fg_fast.  With
// fg_fast == nullptr it is a plain minimise().
MinResult minimise_refined(const FGFun* fg_fast, const FGFun& fg_exact,
                           const std::vector<double>& x0, const std::vector<double>& step,
                           const std::vector<double>& lo, const std::vector<double>& hi,
                           const MinOpts& opt);

}  // namespace gfi
