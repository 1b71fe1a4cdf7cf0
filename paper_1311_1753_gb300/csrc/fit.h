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
};

struct MinResult {
  std::vector<double> x, err, cov;
  double fval = 0.0, edm = 0.0;
  int calls = 0, iters = 0;
  bool converged = false;
  int status = 0;  // GF_OK / GF_ENOCONV / evaluation error code
};

// f(x, g) -> status; x in external units; g (same length) filled with df/dx.
using FGFun = std::function<int(const std::vector<double>&, double&, std::vector<double>&)>;

MinResult minimise(const FGFun& fg, const std::vector<double>& x0, const std::vector<double>& step,
                   const std::vector<double>& lo, const std::vector<double>& hi,
                   const MinOpts& opt);

}  // namespace gfi
