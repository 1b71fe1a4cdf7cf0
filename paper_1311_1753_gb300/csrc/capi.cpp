// capi.cpp -- the C ABI (include/gf.h): contexts, variables, PDF nodes, datasets, the
// PDF-tree compiler and the evaluation path.
//
// The paper's FitManager hands MINUIT a function that copies the parameters to the
// device, runs the per-event evaluate/metric over all events and returns the reduced
// sum (Sec. 2).  Here one evaluation is: one host->device copy of theta, one or two
// kernel launches (normalisation, then the event stream whose last block finishes the
// deterministic reduction), one device->host copy of 1 + n_free doubles.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"
#include "leafrec.h"

using namespace gfi;

namespace gfi {

int set_error(gf_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

static int cuda_fail(gf_ctx* ctx, cudaError_t e, const char* where) {
  cudaGetLastError();  // clear the (non-sticky) error so later calls do not report it
  return set_error(ctx, GF_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

// ---- Weideman coefficients --------------------------------------------------------------
// a_n = (1/2pi) Int_{-pi}^{pi} f(theta) e^{-i n theta} d theta with
// f = (L^2 + t^2) e^{-t^2}, t = L tan(theta/2): a periodic smooth function, so the
// midpoint rule on M points converges faster than any power of 1/M.
static void weideman_coeffs(int N, double L, double* a) {
  const int M = 16 * N;
  const double pi = 3.14159265358979323846;
  for (int n = 0; n <= N; ++n) a[n] = 0.0;
  for (int k = 0; k < M; ++k) {
    const double th = -pi + 2.0 * pi * (k + 0.5) / M;
    const double t = L * std::tan(0.5 * th);
    const double f = (L * L + t * t) * std::exp(-t * t);
    for (int n = 0; n <= N; ++n) a[n] += f * std::cos(n * th);
  }
  for (int n = 0; n <= N; ++n) a[n] /= M;
}

const WeidCoef& weideman() {
  static WeidCoef W;
  static std::once_flag once;
  std::call_once(once, [] {
    const double L = std::pow(2.0, -0.25) * std::sqrt((double)kWeidN);
    double a[kWeidN + 1];
    weideman_coeffs(kWeidN, L, a);
    W.Lhi = (float)L;
    W.Llo = (float)(L - (double)W.Lhi);
    for (int n = 0; n <= kWeidN; ++n) {
      W.ahi[n] = (float)a[n];
      W.alo[n] = (float)(a[n] - (double)W.ahi[n]);
    }
  });
  return W;
}

int nfree(const gf_ctx* ctx) {
  int n = 0;
  for (auto& p : ctx->pars) n += p.fixed ? 0 : 1;
  return n;
}

}  // namespace gfi

// ---- small helpers ------------------------------------------------------------------------------
static bool valid_par(gf_ctx* c, int p) { return p >= 0 && p < (int)c->pars.size(); }
static bool valid_obs(gf_ctx* c, int o) { return o >= 0 && o < (int)c->obs.size(); }
static bool valid_node(gf_ctx* c, int n) { return n >= 0 && n < (int)c->nodes.size(); }

static int add_node(gf_ctx* ctx, NodeDef&& nd, int* node) {
  if (!node) return set_error(ctx, GF_EINVAL, "node output pointer is NULL");
  ctx->nodes.push_back(std::move(nd));
  *node = (int)ctx->nodes.size() - 1;
  ctx->compiled = false;
  return GF_OK;
}

static int leaf(gf_ctx* ctx, int type, int obs, std::vector<int> pars, int* node) {
  if (!ctx) return GF_EINVAL;
  if (!valid_obs(ctx, obs)) return set_error(ctx, GF_EINVAL, "unknown observable id");
  for (int p : pars)
    if (!valid_par(ctx, p)) return set_error(ctx, GF_EINVAL, "unknown parameter id");
  NodeDef nd;
  nd.type = type;
  nd.obs = obs;
  nd.pars = std::move(pars);
  nd.nbx = (type == N_VOIGT || type == N_THRESH) ? 10000 : 0;
  return add_node(ctx, std::move(nd), node);
}

// ---- device memory ------------------------------------------------------------------------------
static void free_dev(gf_ctx* ctx) {
  DevState& d = ctx->dev;
  if (d.copy_stream) {  // a prefetch may still be copying into the staging buffers
    cudaStreamSynchronize(d.copy_stream);
    cudaStreamSynchronize(d.check_stream);
    cudaStreamDestroy(d.copy_stream);
    cudaStreamDestroy(d.check_stream);
  }
  for (int q = 0; q < DevState::kStage; ++q) {
    if (d.ev_copied[q]) cudaEventDestroy(d.ev_copied[q]);
    if (d.ev_staged[q]) cudaEventDestroy(d.ev_staged[q]);
    for (double* p : d.stage[q]) cudaFree(p);
  }
  if (d.ev_free) cudaEventDestroy(d.ev_free);
  if (d.owns_cols)
    for (double* p : d.cols) cudaFree(p);
  d.cols.clear();
  d.owns_cols = false;
  cudaFree(d.theta);
  cudaFree(d.derived);
  cudaFree(d.sbtab);
  cudaFree(d.partials);
  cudaFree(d.partials2);
  cudaFree(d.counters);
  cudaFree(d.norm_out);
  cudaFree(d.inside);
  cudaFree(d.grid_cols);
  cudaFree(d.gram);
  cudaFree(d.ev_cache);
  cudaFree(d.ev_cache64);
  cudaFree(d.fcols);
  cudaFree(d.todo);
  if (d.h_theta) cudaFreeHost(d.h_theta);
  if (d.h_result) cudaFreeHost(d.h_result);
  if (d.ev0) cudaEventDestroy(d.ev0);
  if (d.ev1) cudaEventDestroy(d.ev1);
  if (d.evm) cudaEventDestroy(d.evm);
  cudaFree(d.tick_desc);
  cudaFree(d.prog);
  cudaFree(d.perm);
  cudaFree(d.bw);
  cudaFree(d.bs2);
  cudaFree(d.tddp_cache);
  cudaFree(d.tddp_gcols);
  cudaFree(d.tddp_gram);
  cudaFree(d.tddp_dcache);
  cudaFree(d.tddp_normd);
  for (void* p : d.conv_bufs) cudaFree(p);
  for (void* p : d.gn_bufs) cudaFree(p);
  for (auto& g : d.graph)
    if (g) cudaGraphExecDestroy(g);
  d = DevState();
}

// ---- C ABI: context -------------------------------------------------------------------------------
extern "C" {

namespace {
// Tables and kernel attributes are set up once per device, with that device current,
// before any of the context's work can be captured into a graph.  A failed upload or
// attribute call fails the context's creation (the kernels would otherwise read zero
// tables).
std::mutex g_prep_mu;
bool g_prepared[64] = {false};
cudaError_t prepare_device(int device) {
  std::lock_guard<std::mutex> lk(g_prep_mu);
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  if (g_prepared[device]) return cudaSuccess;
  cudaError_t e = gfi::prepare_kernels_1d();
  if (e == cudaSuccess) e = gfi::prepare_kernels_dalitz();
  if (e == cudaSuccess) e = gfi::prepare_kernels_sigbkg();
  if (e == cudaSuccess) e = gfi::noalloc_preload();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  g_prepared[device] = true;
  return cudaSuccess;
}
}  // namespace

int gf_create(gf_ctx** out, int device, int precision) {
  if (!out) return GF_EINVAL;
  *out = nullptr;
  if (precision != GF_FP64 && precision != GF_MIXED) return GF_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return GF_ECUDA;
  }
  gf_ctx* ctx = new (std::nothrow) gf_ctx();
  if (!ctx) return GF_ENOMEM;
  ctx->device = device;
  ctx->precision = precision;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return GF_ECUDA;
  }
  ctx->stream = ctx->own_stream;
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  weideman();
  const cudaError_t pe = prepare_device(device);
  if (pe != cudaSuccess) {
    cudaStreamDestroy(ctx->own_stream);
    delete ctx;
    return GF_ECUDA;
  }
  *out = ctx;
  return GF_OK;
}

int gf_destroy(gf_ctx* ctx) {
  if (!ctx) return GF_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_dev(ctx);
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  delete ctx;
  return GF_OK;
}

int gf_set_stream(gf_ctx* ctx, void* stream) {
  if (!ctx) return GF_EINVAL;
  ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
  return GF_OK;
}

const char* gf_strerror(int code) {
  switch (code) {
    case GF_OK: return "ok";
    case GF_EINVAL: return "invalid argument";
    case GF_ENOMEM: return "out of memory";
    case GF_ECUDA: return "CUDA runtime error";
    case GF_ENONFINITE: return "non-finite likelihood (some P_i <= 0 or not finite)";
    case GF_ENOCONV: return "minimiser did not converge";
    case GF_ETIMEOUT: return "timed out";
    case GF_ESTATE: return "call out of order";
  }
  return "unknown status";
}

int gf_last_error(gf_ctx* ctx, char* buf, size_t n) {
  if (!ctx || !buf || n == 0) return GF_EINVAL;
  std::snprintf(buf, n, "%s", ctx->err.c_str());
  return GF_OK;
}

// ---- variables ---------------------------------------------------------------------------------------
int gf_observable(gf_ctx* ctx, const char* name, double lo, double hi, int* id) {
  if (!ctx || !id) return GF_EINVAL;
  if (!(lo < hi) || !std::isfinite(lo) || !std::isfinite(hi))
    return set_error(ctx, GF_EINVAL, "observable needs finite lo < hi");
  ctx->obs.push_back({name ? name : "", lo, hi});
  *id = (int)ctx->obs.size() - 1;
  return GF_OK;
}

int gf_parameter(gf_ctx* ctx, const char* name, double init, double step, double lo, double hi,
                 int* id) {
  if (!ctx || !id) return GF_EINVAL;
  if (!std::isfinite(init) || !(step > 0) || !std::isfinite(step))
    return set_error(ctx, GF_EINVAL, "parameter needs a finite value and a step > 0");
  if (!(lo == 0 && hi == 0)) {
    if (!(lo < hi)) return set_error(ctx, GF_EINVAL, "parameter limits need lo < hi");
    if (init < lo || init > hi) return set_error(ctx, GF_EINVAL, "initial value outside limits");
  }
  ctx->pars.push_back({name ? name : "", init, step, lo, hi, false});
  *id = (int)ctx->pars.size() - 1;
  ctx->compiled = false;
  return GF_OK;
}

int gf_set_fixed(gf_ctx* ctx, int par, int fixed) {
  if (!ctx || !valid_par(ctx, par)) return GF_EINVAL;
  if (ctx->pars[par].fixed != (fixed != 0)) {
    ctx->pars[par].fixed = fixed != 0;
    ctx->compiled = false;
  }
  return GF_OK;
}

int gf_set_value(gf_ctx* ctx, int par, double value) {
  if (!ctx || !valid_par(ctx, par) || !std::isfinite(value)) return GF_EINVAL;
  const ParDef& p = ctx->pars[par];
  if (!(p.lo == 0 && p.hi == 0) && (value < p.lo || value > p.hi))
    return set_error(ctx, GF_EINVAL, "value outside the parameter's limits");
  ctx->pars[par].value = value;
  return GF_OK;
}

int gf_get_value(gf_ctx* ctx, int par, double* value) {
  if (!ctx || !valid_par(ctx, par) || !value) return GF_EINVAL;
  *value = ctx->pars[par].value;
  return GF_OK;
}

int gf_free_params(gf_ctx* ctx, int* n, int* ids) {
  if (!ctx || !n) return GF_EINVAL;
  int k = 0;
  for (int i = 0; i < (int)ctx->pars.size(); ++i)
    if (!ctx->pars[i].fixed) {
      if (ids) ids[k] = i;
      ++k;
    }
  *n = k;
  return GF_OK;
}

// ---- PDF nodes ----------------------------------------------------------------------------------------
int gf_pdf_exp(gf_ctx* ctx, int obs, int alpha, int* node) {
  return leaf(ctx, N_EXP, obs, {alpha}, node);
}
int gf_pdf_gauss(gf_ctx* ctx, int obs, int mu, int sigma, int* node) {
  return leaf(ctx, N_GAUSS, obs, {mu, sigma}, node);
}
int gf_pdf_voigt(gf_ctx* ctx, int obs, int mu, int sigma, int width, int* node) {
  return leaf(ctx, N_VOIGT, obs, {mu, sigma, width}, node);
}
int gf_pdf_threshold(gf_ctx* ctx, int obs, int x0, int power, int c, int* node) {
  return leaf(ctx, N_THRESH, obs, {x0, power, c}, node);
}
int gf_pdf_poly(gf_ctx* ctx, int obs, int ncoef, const int* coefs, int* node) {
  if (!ctx) return GF_EINVAL;
  if (ncoef < 1 || ncoef > kMaxLocal || !coefs)
    return set_error(ctx, GF_EINVAL, "polynomial needs 1..8 coefficients");
  return leaf(ctx, N_POLY, obs, std::vector<int>(coefs, coefs + ncoef), node);
}

int gf_pdf_relbw(gf_ctx* ctx, int obs, int dm0, int gamma0, int shift, int ma, int mb,
                 int radius, int spin, int* node) {
  if (!ctx) return GF_EINVAL;
  if (spin < 0 || spin > 2) return set_error(ctx, GF_EINVAL, "relbw: spin 0, 1 or 2");
  const int rc = leaf(ctx, N_RELBW, obs, {dm0, gamma0, shift, ma, mb, radius}, node);
  if (rc == GF_OK) ctx->nodes[*node].aux = spin;
  return rc;
}

int gf_pdf_conv(gf_ctx* ctx, int obs, int model, int resolution, int* node) {
  if (!ctx) return GF_EINVAL;
  if (!valid_obs(ctx, obs) || !valid_node(ctx, model) || !valid_node(ctx, resolution) ||
      model == resolution)
    return set_error(ctx, GF_EINVAL, "ConvolutionPdf: bad observable or nodes");
  for (int c : {model, resolution}) {
    const int t = ctx->nodes[c].type;
    if (t == N_DALITZ || t == N_CONV)
      return set_error(ctx, GF_EINVAL, "ConvolutionPdf: model and resolution are 1D, unconvolved");
  }
  NodeDef nd;
  nd.type = N_CONV;
  nd.obs = obs;
  nd.nbx = 1000;
  nd.children = {model, resolution};
  return add_node(ctx, std::move(nd), node);
}

int gf_pdf_mapped(gf_ctx* ctx, int obs, int n, const int* nodes, const int* bounds, int* node) {
  if (!ctx) return GF_EINVAL;
  if (!valid_obs(ctx, obs) || n < 2 || n > 4 || !nodes || !bounds)
    return set_error(ctx, GF_EINVAL, "MappedPdf: 2..4 components over one observable");
  NodeDef nd;
  nd.type = N_MAPPED;
  nd.obs = obs;
  for (int k = 0; k < n; ++k) {
    if (!valid_node(ctx, nodes[k]) || ctx->nodes[nodes[k]].type == N_DALITZ)
      return set_error(ctx, GF_EINVAL, "MappedPdf: unknown or non-1D component");
    nd.children.push_back(nodes[k]);
  }
  for (int k = 0; k < n - 1; ++k) {
    if (!valid_par(ctx, bounds[k])) return set_error(ctx, GF_EINVAL, "MappedPdf: unknown boundary id");
    nd.pars.push_back(bounds[k]);
  }
  return add_node(ctx, std::move(nd), node);
}

int gf_pdf_composite(gf_ctx* ctx, int obs, int core, int shell, int* node) {
  if (!ctx) return GF_EINVAL;
  if (!valid_obs(ctx, obs) || !valid_node(ctx, core) || !valid_node(ctx, shell) || core == shell)
    return set_error(ctx, GF_EINVAL, "CompositePdf: bad observable or nodes");
  const int ct = ctx->nodes[core].type, st = ctx->nodes[shell].type;
  if (!(ct >= N_EXP && ct <= N_RELBW) || ctx->nodes[core].obs != obs)
    return set_error(ctx, GF_EINVAL, "CompositePdf: the core is a leaf over the observable");
  if (st != N_EXP && st != N_GAUSS && st != N_POLY)
    return set_error(ctx, GF_EINVAL, "CompositePdf: the shell is an exponential, Gaussian or polynomial");
  NodeDef nd;
  nd.type = N_COMPOSITE;
  nd.obs = obs;
  nd.children = {core, shell};
  return add_node(ctx, std::move(nd), node);
}

int gf_pdf_add(gf_ctx* ctx, int n, const int* nodes, const int* fracs, int* node) {
  if (!ctx) return GF_EINVAL;
  if (n < 2 || n > kMaxLocal || !nodes || !fracs)
    return set_error(ctx, GF_EINVAL, "AddPdf needs 2..8 components and n-1 fractions");
  NodeDef nd;
  nd.type = N_ADD;
  for (int k = 0; k < n; ++k) {
    if (!valid_node(ctx, nodes[k]) || ctx->nodes[nodes[k]].type == N_DALITZ)
      return set_error(ctx, GF_EINVAL, "AddPdf: unknown or non-1D component");
    nd.children.push_back(nodes[k]);
  }
  for (int k = 0; k < n - 1; ++k) {
    if (!valid_par(ctx, fracs[k])) return set_error(ctx, GF_EINVAL, "AddPdf: unknown fraction id");
    nd.pars.push_back(fracs[k]);
  }
  return add_node(ctx, std::move(nd), node);
}

int gf_pdf_prod(gf_ctx* ctx, int n, const int* nodes, int* node) {
  if (!ctx) return GF_EINVAL;
  if (n < 2 || n > kMaxLocal || !nodes)
    return set_error(ctx, GF_EINVAL, "ProdPdf needs 2..8 factors");
  NodeDef nd;
  nd.type = N_PROD;
  for (int k = 0; k < n; ++k) {
    if (!valid_node(ctx, nodes[k]) || ctx->nodes[nodes[k]].type == N_DALITZ)
      return set_error(ctx, GF_EINVAL, "ProdPdf: unknown or non-1D factor");
    nd.children.push_back(nodes[k]);
  }
  return add_node(ctx, std::move(nd), node);
}

int gf_pdf_dalitz(gf_ctx* ctx, int obs12, int obs13, const gf_dalitz_kin* kin, int nres,
                  const gf_resonance* res, int* node) {
  if (!ctx) return GF_EINVAL;
  if (!valid_obs(ctx, obs12) || !valid_obs(ctx, obs13) || obs12 == obs13 || !kin)
    return set_error(ctx, GF_EINVAL, "Dalitz: bad observables or kinematics");
  if (nres < 0 || nres > kMaxRes || (nres > 0 && !res))
    return set_error(ctx, GF_EINVAL, "Dalitz: 0..12 resonances");
  if (!(kin->M > kin->m1 + kin->m2 + kin->m3) || !(kin->m1 > 0) || !(kin->m2 > 0) ||
      !(kin->m3 > 0) || !(kin->R >= 0))
    return set_error(ctx, GF_EINVAL, "Dalitz: masses must satisfy M > m1 + m2 + m3 > 0");
  NodeDef nd;
  nd.type = N_DALITZ;
  nd.obs = obs12;
  nd.obs2 = obs13;
  nd.kin = *kin;
  nd.nbx = 512;
  nd.nby = 512;
  for (int r = 0; r < nres; ++r) {
    const gf_resonance& R = res[r];
    if (R.channel < 0 || R.channel > 2 || R.spin < 0 || R.spin > 2 || !valid_par(ctx, R.mass) ||
        !valid_par(ctx, R.width) || !valid_par(ctx, R.re) || !valid_par(ctx, R.im))
      return set_error(ctx, GF_EINVAL, "Dalitz: bad resonance (channel 0..2, spin 0..2, ids)");
    nd.res.push_back(R);
  }
  return add_node(ctx, std::move(nd), node);
}

int gf_pdf_tddp(gf_ctx* ctx, int obs12, int obs13, int obs_t, int obs_sigt,
                const gf_dalitz_kin* kin, int nres, const gf_resonance* res, int tau, int x,
                int y, int scale, int* node) {
  if (!ctx) return GF_EINVAL;
  int id = -1;
  int rc = gf_pdf_dalitz(ctx, obs12, obs13, kin, nres, res, &id);
  if (rc) return rc;
  NodeDef& nd = ctx->nodes[id];
  if (!valid_obs(ctx, obs_t) || !valid_obs(ctx, obs_sigt) || obs_t == obs_sigt ||
      obs_t == obs12 || obs_t == obs13 || obs_sigt == obs12 || obs_sigt == obs13)
    return set_error(ctx, GF_EINVAL, "time-dependent Dalitz: bad time observables");
  if (!(std::fabs(kin->m1 - kin->m2) <= 1e-12 * kin->m1))
    return set_error(ctx, GF_EINVAL, "time-dependent Dalitz: particles 1 and 2 are CP conjugates (m1 = m2)");
  for (int p : {tau, x, y, scale})
    if (!valid_par(ctx, p)) return set_error(ctx, GF_EINVAL, "time-dependent Dalitz: unknown parameter id");
  nd.type = N_TDDP;
  nd.obs3 = obs_t;
  nd.obs4 = obs_sigt;
  nd.pars = {tau, x, y, scale};
  nd.nbx = nd.nby = 256;
  *node = id;
  return GF_OK;
}

int gf_tddp_sigt_density(gf_ctx* ctx, int node, int b0, int b1, int b2) {
  if (!ctx || !valid_node(ctx, node)) return GF_EINVAL;
  NodeDef& nd = ctx->nodes[node];
  if (nd.type != N_TDDP)
    return set_error(ctx, GF_EINVAL, "sigma_t density: not a time-dependent Dalitz node");
  for (int p : {b0, b1, b2})
    if (!valid_par(ctx, p)) return set_error(ctx, GF_EINVAL, "sigma_t density: unknown parameter id");
  if (!(ctx->obs[nd.obs4].lo > 0.0))
    return set_error(ctx, GF_EINVAL, "sigma_t density: the sigma_t range must be positive");
  nd.pars.resize(4);
  nd.pars.insert(nd.pars.end(), {b0, b1, b2});
  nd.aux = 1;
  ctx->compiled = false;
  return GF_OK;
}

int gf_set_norm_grid(gf_ctx* ctx, int node, int nbins_x, int nbins_y) {
  if (!ctx || !valid_node(ctx, node)) return GF_EINVAL;
  NodeDef& nd = ctx->nodes[node];
  if (nd.type == N_DALITZ || nd.type == N_TDDP) {
    if (nbins_x < 1 || nbins_y < 1 || (int64_t)nbins_x * nbins_y > (1 << 26))
      return set_error(ctx, GF_EINVAL, "Dalitz grid: 1 <= nbx*nby <= 2^26");
    nd.nby = nbins_y;
  } else if (nd.type == N_VOIGT || nd.type == N_THRESH || nd.type == N_RELBW) {
    if (nbins_x < 1 || nbins_x > (1 << 24)) return set_error(ctx, GF_EINVAL, "grid: 1..2^24 bins");
  } else if (nd.type == N_CONV) {
    if (nbins_x < 1 || nbins_x > kConvMaxLattice)
      return set_error(ctx, GF_EINVAL, "convolution lattice: 1..65536 bins");
  } else if (nd.type == N_MAPPED || nd.type == N_COMPOSITE) {
    if (nbins_x < 1 || nbins_x > (1 << 24)) return set_error(ctx, GF_EINVAL, "grid: 1..2^24 bins");
  } else {
    return set_error(ctx, GF_EINVAL, "node has an analytic normalisation");
  }
  nd.nbx = nbins_x;
  ctx->compiled = false;
  ctx->dev.gram_valid = false;
  ctx->dev.mask_built = false;
  return GF_OK;
}

}  // extern "C"

// ---- Dalitz host-side geometry --------------------------------------------------------------------
static void fill_channel(DalitzChannel& c, double M, double ma, double mb, double mc) {
  c.ma2 = ma * ma;
  c.mb2 = mb * mb;
  c.mc2 = mc * mc;
  c.thrA = (ma + mb) * (ma + mb);
  c.thrB = (ma - mb) * (ma - mb);
  c.k1 = (M * M - mc * mc) * (ma * ma - mb * mb);
  c.a2c = 2 * M * M + 2 * mc * mc;
  c.a2k = (M * M - mc * mc) * (M * M - mc * mc);
}

static void dalitz_geometry(const NodeDef& nd, DalitzPlan& D) {
  const gf_dalitz_kin& k = nd.kin;
  D.M = k.M;
  D.m1 = k.m1;
  D.m2 = k.m2;
  D.m3 = k.m3;
  D.M2 = k.M * k.M;
  D.sum_m2 = D.M2 + k.m1 * k.m1 + k.m2 * k.m2 + k.m3 * k.m3;
  D.R2 = k.R * k.R;
  fill_channel(D.ch[0], k.M, k.m1, k.m2, k.m3);
  fill_channel(D.ch[1], k.M, k.m1, k.m3, k.m2);
  fill_channel(D.ch[2], k.M, k.m2, k.m3, k.m1);
  D.nbx = nd.nbx;
  D.nby = nd.nby;
  D.x0 = (k.m1 + k.m2) * (k.m1 + k.m2);
  D.hx = ((k.M - k.m3) * (k.M - k.m3) - D.x0) / nd.nbx;
  D.y0 = (k.m1 + k.m3) * (k.m1 + k.m3);
  D.hy = ((k.M - k.m2) * (k.M - k.m2) - D.y0) / nd.nby;
}

// Same region test as the device (|cos theta_12| <= 1 as S_1^2 <= a2 a3).
static bool dalitz_inside_host(const DalitzPlan& D, double s12, double s13) {
  const double s23 = D.sum_m2 - s12 - s13;
  const DalitzChannel& c = D.ch[0];
  if (!(s12 > c.thrA) || !(s13 > D.ch[1].thrA) || !(s23 > D.ch[2].thrA)) return false;
  const double inv_s = 1.0 / s12;
  const double S1 = s23 - s13 + c.k1 * inv_s;
  const double a2 = s12 - c.a2c + c.a2k * inv_s;
  const double a3 = (s12 - c.thrA) * (s12 - c.thrB) * inv_s;
  return S1 * S1 <= a2 * a3;
}

extern "C" int gf_dalitz_inside(gf_ctx* ctx, int node, int64_t n, const double* s12,
                                const double* s13, int8_t* out) {
  if (!ctx || !valid_node(ctx, node) ||
      (ctx->nodes[node].type != N_DALITZ && ctx->nodes[node].type != N_TDDP) || n < 0 ||
      (n > 0 && (!s12 || !s13 || !out)))
    return GF_EINVAL;
  DalitzPlan D{};
  dalitz_geometry(ctx->nodes[node], D);
  for (int64_t i = 0; i < n; ++i) out[i] = dalitz_inside_host(D, s12[i], s13[i]) ? 1 : 0;
  return GF_OK;
}

// ---- the PDF-tree compiler (1D trees) ------------------------------------------------------------
namespace {

// A ConvolutionPdf found by the compiler: its model and resolution subtrees as programs of
// their own (sharing the main program's leaf and coefficient tables).
struct ConvInfo {
  int node = -1, mcol = -1, ro = -1, slot = -1;
  std::vector<int> loc;  // local parameters (free parameters of both subtrees)
  Program pm{}, pr{};
};

// A MappedPdf or CompositePdf found by the compiler: its body as a program of its own
// (the grid normalisation evaluates it at midpoints), also copied into the main program.
struct GNInfo {
  int node = -1, mcol = -1, slot = -1;
  std::vector<int> loc;
  Program body{};
};

int first_leaf_obs(const gf_ctx* ctx, int id) {
  const NodeDef& nd = ctx->nodes[id];
  if (nd.type >= N_EXP && nd.type <= N_RELBW) return nd.obs;
  return nd.children.empty() ? -1 : first_leaf_obs(ctx, nd.children[0]);
}

struct Compiler {
  gf_ctx* ctx;
  Program& P;
  const std::vector<int>& col_of_obs;  // observable id -> dataset column, -1 if absent
  std::string err;
  int depth = 0, maxdepth = 0;
  // convolutions: instructions of a subtree go to tgt (the main program when null); inside
  // a resolution its residual observable resid_obs maps to column kResidCol; conv_pars
  // collects the parameters of the subtree's leaves and fractions
  Program* tgt = nullptr;
  int resid_obs = -1, conv_mobs = -1;
  std::vector<int>* conv_pars = nullptr;
  std::vector<ConvInfo> convs;
  std::vector<GNInfo> gns;
  bool raw_next = false;  // the next leaf keeps its unnormalised shape (CompositePdf core)

  int need(int id) {
    const NodeDef& nd = ctx->nodes[id];
    if (nd.type == N_MAPPED) return 3;  // component, indicator, running sum
    if (nd.type != N_ADD && nd.type != N_PROD) return 1;
    std::vector<int> nn;
    for (int c : nd.children) nn.push_back(need(c));
    std::sort(nn.rbegin(), nn.rend());
    int m = 0;
    for (size_t k = 0; k < nn.size(); ++k) m = std::max(m, nn[k] + (k > 0 ? 1 : 0));
    return m;
  }
  std::vector<int> ordered(const NodeDef& nd) {
    std::vector<int> idx(nd.children.size());
    for (size_t k = 0; k < idx.size(); ++k) idx[k] = (int)k;
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int a, int b) { return need(nd.children[a]) > need(nd.children[b]); });
    return idx;
  }
  bool emit(const Instr& I) {
    Program& T = tgt ? *tgt : P;
    if (T.n >= kMaxIns) { err = "PDF tree too large (more than 32 instructions)"; return false; }
    T.ins[T.n++] = I;
    if (I.op == OP_LEAF) depth++;
    if (I.op == OP_MUL || I.op == OP_LMUL || I.op == OP_ADD) depth--;
    maxdepth = std::max(maxdepth, depth);
    return true;
  }
  int gidx(int par) const { return ctx->free_pos[par]; }

  // returns 1 for log domain, 0 linear, -1 error
  int walk(int id, std::vector<int>& obs_used) {
    const NodeDef& nd = ctx->nodes[id];
    if (nd.type >= N_EXP && nd.type <= N_RELBW) {
      if (P.nleaf >= kMaxLeaf) { err = "more than 16 leaves"; return -1; }
      if (resid_obs >= 0 && nd.obs != resid_obs) {
        err = "a resolution's leaves must share one residual observable";
        return -1;
      }
      if (conv_mobs >= 0 && nd.obs != conv_mobs) {
        err = "a convolution's model must use the convolution's observable";
        return -1;
      }
      const int col = resid_obs >= 0 ? kResidCol : col_of_obs[nd.obs];
      if (col < 0) { err = "the dataset lacks an observable used by the PDF"; return -1; }
      if (nd.type == N_RELBW)
        for (int k = 2; k < 6; ++k)
          if (gidx(nd.pars[k]) >= 0) {
            err = "relbw: shift, daughter masses and radius must be fixed parameters";
            return -1;
          }
      obs_used.push_back(nd.obs);
      if (conv_pars) conv_pars->insert(conv_pars->end(), nd.pars.begin(), nd.pars.end());
      LeafDesc& L = P.leaf[P.nleaf];
      L = LeafDesc{};
      L.kind = nd.type;  // N_EXP..N_RELBW coincide with L_EXP..L_RELBW
      L.obs = col;
      L.npar = (int)nd.pars.size();
      L.aux = nd.aux | (raw_next ? kRawLeaf : 0);
      for (int k = 0; k < L.npar; ++k) L.par[k] = nd.pars[k];
      L.nbins = (!raw_next && (nd.type == N_VOIGT || nd.type == N_THRESH || nd.type == N_RELBW))
                    ? nd.nbx : 0;
      L.lo = ctx->obs[nd.obs].lo;
      L.hi = ctx->obs[nd.obs].hi;
      Instr I{};
      I.op = OP_LEAF;
      I.kind = nd.type;
      I.obs = col;
      I.slot = P.nleaf;
      I.npar = L.npar;
      for (int k = 0; k < kMaxLocal; ++k) I.gidx[k] = k < L.npar ? gidx(L.par[k]) : -1;
      P.nleaf++;
      if (!emit(I)) return -1;
      return (nd.type == N_EXP || nd.type == N_GAUSS) ? 1 : 0;
    }
    if (nd.type == N_CONV) {
      if (tgt) { err = "ConvolutionPdf nodes cannot be nested"; return -1; }
      if ((int)convs.size() >= kMaxConv) { err = "more than 2 ConvolutionPdf nodes"; return -1; }
      if (P.nleaf >= kMaxLeaf) { err = "more than 16 leaves"; return -1; }
      ConvInfo ci;
      ci.node = id;
      ci.mcol = col_of_obs[nd.obs];
      ci.ro = first_leaf_obs(ctx, nd.children[1]);
      if (ci.mcol < 0) { err = "the dataset lacks the convolution's observable"; return -1; }
      if (ci.ro < 0 || ci.ro == nd.obs) {
        err = "the resolution needs its own residual observable";
        return -1;
      }
      std::vector<int> pars, u;
      conv_pars = &pars;
      const int saved = depth;
      tgt = &ci.pm;
      depth = 0;
      conv_mobs = nd.obs;
      const int dm = walk(nd.children[0], u);
      conv_mobs = -1;
      if (dm < 0) return -1;
      ci.pm.root_log = dm;
      tgt = &ci.pr;
      depth = 0;
      resid_obs = ci.ro;
      const int dr = walk(nd.children[1], u);
      resid_obs = -1;
      tgt = nullptr;
      depth = saved;
      conv_pars = nullptr;
      if (dr < 0) return -1;
      ci.pr.root_log = dr;
      for (int q : pars)
        if (gidx(q) >= 0 && std::find(ci.loc.begin(), ci.loc.end(), q) == ci.loc.end())
          ci.loc.push_back(q);
      if ((int)ci.loc.size() > kMaxLocal) {
        err = "a convolution's model and resolution have more than 8 free parameters";
        return -1;
      }
      LeafDesc& L = P.leaf[P.nleaf];
      L = LeafDesc{};
      L.kind = L_CONV;
      L.obs = ci.mcol;
      L.npar = (int)ci.loc.size();
      for (int k = 0; k < L.npar; ++k) L.par[k] = ci.loc[k];
      L.lo = ctx->obs[nd.obs].lo;
      L.hi = ctx->obs[nd.obs].hi;
      L.aux = (int)convs.size();
      Instr I{};
      I.op = OP_LEAF;
      I.kind = L_CONV;
      I.obs = ci.mcol;
      I.slot = P.nleaf;
      I.npar = L.npar;
      for (int k = 0; k < kMaxLocal; ++k) I.gidx[k] = k < L.npar ? gidx(L.par[k]) : -1;
      ci.slot = P.nleaf++;
      if (!emit(I)) return -1;
      obs_used.push_back(nd.obs);
      convs.push_back(std::move(ci));
      return 0;
    }
    if (nd.type == N_MAPPED || nd.type == N_COMPOSITE) {
      if (tgt) { err = "MappedPdf/CompositePdf nodes cannot be nested"; return -1; }
      if ((int)gns.size() >= kMaxGNorm) { err = "more than 2 MappedPdf/CompositePdf nodes"; return -1; }
      GNInfo gi;
      gi.node = id;
      gi.mcol = col_of_obs[nd.obs];
      if (gi.mcol < 0) { err = "the dataset lacks the node's observable"; return -1; }
      std::vector<int> pars, u;
      conv_pars = &pars;
      const int saved = depth;
      tgt = &gi.body;
      depth = 0;
      auto leaf_slot = [&]() -> int {
        if (P.nleaf >= kMaxLeaf) { err = "more than 16 leaves"; return -1; }
        P.leaf[P.nleaf] = LeafDesc{};
        return P.nleaf++;
      };
      if (nd.type == N_MAPPED) {
        const int nc = (int)nd.children.size();
        for (int k = 0; k < nc; ++k) {
          const int dk = walk(nd.children[k], u);
          if (dk < 0) return -1;
          if (dk == 1) {
            Instr T{};
            T.op = OP_TOLIN;
            if (!emit(T)) return -1;
          }
          const int sl = leaf_slot();
          if (sl < 0) return -1;
          LeafDesc& L = P.leaf[sl];
          L.kind = L_IND;
          L.obs = gi.mcol;
          L.lo = ctx->obs[nd.obs].lo;
          L.hi = ctx->obs[nd.obs].hi;
          if (k > 0) L.par[L.npar++] = nd.pars[k - 1];
          if (k < nc - 1) L.par[L.npar++] = nd.pars[k];
          L.aux = (k > 0 ? 1 : 0) | (k < nc - 1 ? 2 : 0);
          for (int q = 0; q < L.npar; ++q)
            if (gidx(L.par[q]) >= 0) { err = "MappedPdf boundaries must be fixed"; return -1; }
          Instr I{};
          I.op = OP_LEAF;
          I.kind = L_IND;
          I.obs = gi.mcol;
          I.slot = sl;
          for (int q = 0; q < kMaxLocal; ++q) I.gidx[q] = -1;
          Instr M{};
          M.op = OP_MUL;
          if (!emit(I) || !emit(M)) return -1;
          if (k > 0) {
            Instr A{};
            A.op = OP_ADD;
            if (!emit(A)) return -1;
          }
        }
      } else {
        raw_next = true;
        const int dc = walk(nd.children[0], u);
        raw_next = false;
        if (dc < 0) return -1;
        if (dc == 1) {
          Instr T{};
          T.op = OP_TOLIN;
          if (!emit(T)) return -1;
        }
        const NodeDef& sh = ctx->nodes[nd.children[1]];
        const int sl = leaf_slot();
        if (sl < 0) return -1;
        LeafDesc& L = P.leaf[sl];
        L.kind = sh.type;
        L.obs = gi.mcol;  // unused: the shell reads the core's value
        L.npar = (int)sh.pars.size();
        for (int k = 0; k < L.npar; ++k) L.par[k] = sh.pars[k];
        L.lo = ctx->obs[sh.obs].lo;
        L.hi = ctx->obs[sh.obs].hi;
        L.aux = kRawLeaf;
        pars.insert(pars.end(), sh.pars.begin(), sh.pars.end());
        Instr C{};
        C.op = OP_COMPOSE;
        C.kind = sh.type;
        C.slot = sl;
        C.npar = L.npar;
        for (int k = 0; k < kMaxLocal; ++k) C.gidx[k] = k < L.npar ? gidx(L.par[k]) : -1;
        if (!emit(C)) return -1;
      }
      tgt = nullptr;
      depth = saved;
      conv_pars = nullptr;
      for (int q : pars)
        if (gidx(q) >= 0 && std::find(gi.loc.begin(), gi.loc.end(), q) == gi.loc.end())
          gi.loc.push_back(q);
      if ((int)gi.loc.size() > kMaxLocal) {
        err = "a MappedPdf/CompositePdf has more than 8 free parameters";
        return -1;
      }
      const int gs = leaf_slot();
      if (gs < 0) return -1;
      LeafDesc& G = P.leaf[gs];
      G.kind = L_GNORM;
      G.obs = gi.mcol;
      G.npar = (int)gi.loc.size();
      for (int k = 0; k < G.npar; ++k) G.par[k] = gi.loc[k];
      G.lo = ctx->obs[nd.obs].lo;
      G.hi = ctx->obs[nd.obs].hi;
      gi.slot = gs;
      for (int pc = 0; pc < gi.body.n; ++pc)
        if (!emit(gi.body.ins[pc])) return -1;
      Instr Nm{};
      Nm.op = OP_GNORM;
      Nm.slot = gs;
      Nm.npar = G.npar;
      for (int k = 0; k < kMaxLocal; ++k) Nm.gidx[k] = k < G.npar ? gidx(G.par[k]) : -1;
      if (!emit(Nm)) return -1;
      obs_used.push_back(nd.obs);
      gns.push_back(std::move(gi));
      return 0;
    }
    if (nd.type == N_PROD) {
      // factors must use distinct observables (ProdPdf of Listing 2)
      std::vector<std::vector<int>> used(nd.children.size());
      std::vector<int> dom(nd.children.size());
      bool all_log = true;
      // decide the domain first: log if every factor is naturally log
      for (int c : nd.children) all_log = all_log && natural_log(c);
      auto ord = ordered(nd);
      for (size_t k = 0; k < ord.size(); ++k) {
        const int j = ord[k];
        int d = walk(nd.children[j], used[j]);
        if (d < 0) return -1;
        if (!all_log && d == 1) {
          Instr T{};
          T.op = OP_TOLIN;
          if (!emit(T)) return -1;
        }
        if (k > 0) {
          Instr M{};
          M.op = all_log ? OP_LMUL : OP_MUL;
          if (!emit(M)) return -1;
        }
      }
      for (size_t a = 0; a < used.size(); ++a)
        for (size_t b = a + 1; b < used.size(); ++b)
          for (int x : used[a])
            for (int y : used[b])
              if (x == y) { err = "ProdPdf factors share an observable"; return -1; }
      for (auto& u : used) obs_used.insert(obs_used.end(), u.begin(), u.end());
      return all_log ? 1 : 0;
    }
    if (nd.type == N_ADD) {
      const int nc = (int)nd.children.size();
      auto ord = ordered(nd);
      for (int k = 0; k < nc; ++k) {
        const int j = ord[k];
        int d = walk(nd.children[j], obs_used);
        if (d < 0) return -1;
        if (d == 1) {
          Instr T{};
          T.op = OP_TOLIN;
          if (!emit(T)) return -1;
        }
        if (P.ncoef >= kMaxCoef) { err = "more than 16 fraction coefficients"; return -1; }
        CoefDesc& C = P.coef[P.ncoef];
        C = CoefDesc{};
        Instr S{};
        S.op = OP_SCALE;
        S.slot = P.ncoef;
        if (j < nc - 1) {
          C.sign = 1;
          C.n = 1;
          C.par[0] = nd.pars[j];
        } else {
          C.sign = -1;
          C.n = nc - 1;
          for (int q = 0; q < nc - 1; ++q) C.par[q] = nd.pars[q];
        }
        if (conv_pars) conv_pars->insert(conv_pars->end(), C.par, C.par + C.n);
        S.kind = C.sign;
        S.npar = C.n;
        for (int q = 0; q < kMaxLocal; ++q) S.gidx[q] = q < C.n ? gidx(C.par[q]) : -1;
        P.ncoef++;
        if (!emit(S)) return -1;
        if (k > 0) {
          Instr A{};
          A.op = OP_ADD;
          if (!emit(A)) return -1;
        }
      }
      return 0;
    }
    err = "a Dalitz node can only be the root of its own PDF";
    return -1;
  }
  bool natural_log(int id) {
    const NodeDef& nd = ctx->nodes[id];
    if (nd.type == N_EXP || nd.type == N_GAUSS) return true;
    if (nd.type == N_PROD) {
      for (int c : nd.children)
        if (!natural_log(c)) return false;
      return true;
    }
    return false;
  }
};

// An AddPdf whose children are leaves compiles to K x [LEAF, (TOLIN), SCALE, (ADD)]; the
// event kernel then evaluates P = sum_k c_k L_k directly (each leaf with at most
// kMixLocal parameters, K <= kMixMax), otherwise the program runs on the stack machine.
static void detect_mixture(Program& P) {
  P.mix = 0;
  if (P.root_log) return;
  int pc = 0, K = 0;
  int lf[kMixMax], lg[kMixMax], sc[kMixMax];
  while (pc < P.n) {
    if (K >= kMixMax) return;
    // the basic leaves only (the mixture kernel holds no code for the others)
    if (P.ins[pc].op != OP_LEAF || P.ins[pc].npar > kMixLocal || P.ins[pc].kind > L_POLY) return;
    lf[K] = pc++;
    lg[K] = 0;
    if (pc < P.n && P.ins[pc].op == OP_TOLIN) {
      lg[K] = 1;
      ++pc;
    }
    if (pc >= P.n || P.ins[pc].op != OP_SCALE) return;
    sc[K] = pc++;
    if (K > 0) {
      if (pc >= P.n || P.ins[pc].op != OP_ADD) return;
      ++pc;
    }
    ++K;
  }
  if (K < 2) return;
  P.mix = K;
  for (int k = 0; k < K; ++k) {
    P.mix_leaf[k] = lf[k];
    P.mix_log[k] = lg[k];
    P.mix_scale[k] = sc[k];
  }
}

// A log-domain product of exponential and Gaussian leaves (LEAF, then (LEAF, LMUL) x
// (K - 1), K <= kLogLeaf, over at most two observables) runs on the direct log-sum kernel.
static void detect_logsum(Program& P) {
  P.logsum = 0;
  if (!P.root_log || P.nobs > 2 || P.nleaf < 1 || P.nleaf > kLogLeaf || P.n != 2 * P.nleaf - 1)
    return;
  for (int pc = 0; pc < P.n; ++pc) {
    const Instr& I = P.ins[pc];
    const bool leaf_slot = pc == 0 || (pc % 2) == 1;
    if (leaf_slot) {
      if (I.op != OP_LEAF || (I.kind != L_EXP && I.kind != L_GAUSS) ||
          I.slot != (pc == 0 ? 0 : (pc + 1) / 2) || I.obs > 1)
        return;
    } else if (I.op != OP_LMUL) {
      return;
    }
  }
  for (int l = 0; l < P.nleaf; ++l)
    if (P.leaf[l].nbins > 0) return;
  P.logsum = 1;
}

// An AddPdf of one Voigtian and one threshold leaf over the same observable (the paper's
// signal + background line shape, Sec. 4) runs on its own kernel (k_sigbkg.cu).
static bool detect_sigbkg(const Program& P, SigBkgDesc& D) {
  if (P.mix != 2 || P.binned) return false;
  int kv = -1, kt = -1;
  for (int k = 0; k < 2; ++k) {
    const Instr& I = P.ins[P.mix_leaf[k]];
    if (I.kind == L_VOIGT && kv < 0) kv = k;
    else if (I.kind == L_THRESH && kt < 0) kt = k;
  }
  if (kv < 0 || kt < 0) return false;
  const Instr& V = P.ins[P.mix_leaf[kv]];
  const Instr& T = P.ins[P.mix_leaf[kt]];
  const Instr& SV = P.ins[P.mix_scale[kv]];
  const Instr& ST = P.ins[P.mix_scale[kt]];
  if (V.obs != T.obs || P.mix_log[kv] || P.mix_log[kt] || V.npar != 3 || T.npar != 3 ||
      SV.npar != 1 || ST.npar != 1 || P.leaf[V.slot].nbins <= 0 || P.leaf[T.slot].nbins <= 0)
    return false;
  D = SigBkgDesc{};
  D.slot_v = V.slot;
  D.slot_t = T.slot;
  D.cslot_v = SV.slot;
  D.cslot_t = ST.slot;
  for (int j = 0; j < 3; ++j) {
    D.gv[j] = V.gidx[j];
    D.gt[j] = T.gidx[j];
  }
  D.fpos_v = SV.gidx[0];
  D.fpos_t = ST.gidx[0];
  D.fsgn_v = SV.kind;
  D.fsgn_t = ST.kind;
  D.nfree = P.nfree;
  return true;
}

// Device tables of every convolution (freed and rebuilt at each compilation).
static void free_convs(DevState& d) {
  for (void* p : d.conv_bufs) cudaFree(p);
  d.conv_bufs.clear();
  d.nconv = 0;
  for (auto& c : d.conv_desc) c = nullptr;
}

static int setup_convs(gf_ctx* ctx, std::vector<ConvInfo>& convs) {
  DevState& d = ctx->dev;
  free_convs(d);
  const Program& P = ctx->prog;
  for (size_t c = 0; c < convs.size(); ++c) {
    ConvInfo& ci = convs[c];
    const NodeDef& nd = ctx->nodes[ci.node];
    for (Program* sp : {&ci.pm, &ci.pr}) {  // the subtrees share the main tables
      sp->nleaf = P.nleaf;
      sp->ncoef = P.ncoef;
      sp->nfree = P.nfree;
      sp->nobs = P.nobs;
      std::copy(P.leaf, P.leaf + kMaxLeaf, sp->leaf);
      std::copy(P.coef, P.coef + kMaxCoef, sp->coef);
    }
    ConvDesc h{};
    h.L = nd.nbx;
    h.lo = ctx->obs[nd.obs].lo;
    h.h = (ctx->obs[nd.obs].hi - h.lo) / h.L;
    h.kmin = (int)std::ceil(ctx->obs[ci.ro].lo / h.h - 1e-9);
    h.kmax = (int)std::floor(ctx->obs[ci.ro].hi / h.h + 1e-9);
    h.K = h.kmax - h.kmin + 1;
    if (h.K < 1 || h.K > kConvMaxOffsets)
      return set_error(ctx, GF_EINVAL,
                       "convolution: 1..8193 lattice steps must fit the residual range");
    h.J = h.L + h.K;
    h.nloc = (int)ci.loc.size();
    h.slot = ci.slot;
    h.mcol = ci.mcol;
    for (int l = 0; l < h.nloc; ++l) h.loc2free[l] = ctx->free_pos[ci.loc[l]];
    const int nq = 1 + h.nloc;
    auto alloc = [&](size_t bytes) -> void* {
      void* p = nullptr;
      if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      d.conv_bufs.push_back(p);
      return p;
    };
    Program* pm = static_cast<Program*>(alloc(sizeof(Program)));
    Program* pr = static_cast<Program*>(alloc(sizeof(Program)));
    h.mt = static_cast<float2*>(alloc(sizeof(float2) * nq * (size_t)h.J));
    h.rt = static_cast<float2*>(alloc(sizeof(float2) * nq * (size_t)h.K));
    h.ct = static_cast<double*>(alloc(sizeof(double) * nq * (size_t)(h.L + 1)));
    h.partials = static_cast<double*>(alloc(sizeof(double) * nq * (size_t)(h.L + 1)));
    h.counter = static_cast<unsigned*>(alloc(sizeof(unsigned)));
    ConvDesc* dd = static_cast<ConvDesc*>(alloc(sizeof(ConvDesc)));
    if (!pm || !pr || !h.mt || !h.rt || !h.ct || !h.partials || !h.counter || !dd) {
      free_convs(d);
      return set_error(ctx, GF_ENOMEM, "device allocation of the convolution tables failed");
    }
    h.pm = pm;
    h.pr = pr;
    CK(cudaMemcpyAsync(pm, &ci.pm, sizeof(Program), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(pr, &ci.pr, sizeof(Program), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(h.counter, 0, sizeof(unsigned), ctx->stream));
    CK(cudaMemcpyAsync(dd, &h, sizeof(ConvDesc), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    d.conv_host[c] = h;
    d.conv_desc[c] = dd;
    d.nconv = (int)c + 1;
  }
  return GF_OK;
}

static void free_gnorms(DevState& d) {
  for (void* p : d.gn_bufs) cudaFree(p);
  d.gn_bufs.clear();
  d.ngn = 0;
  for (auto& g : d.gn_desc) g = nullptr;
}

static int setup_gnorms(gf_ctx* ctx, std::vector<GNInfo>& gns) {
  DevState& d = ctx->dev;
  free_gnorms(d);
  const Program& P = ctx->prog;
  for (size_t g = 0; g < gns.size(); ++g) {
    GNInfo& gi = gns[g];
    const NodeDef& nd = ctx->nodes[gi.node];
    Program& B = gi.body;
    B.nleaf = P.nleaf;
    B.ncoef = P.ncoef;
    B.nfree = P.nfree;
    B.nobs = P.nobs;
    std::copy(P.leaf, P.leaf + kMaxLeaf, B.leaf);
    std::copy(P.coef, P.coef + kMaxCoef, B.coef);
    GNormDesc h{};
    h.nbins = nd.nbx;
    h.lo = ctx->obs[nd.obs].lo;
    h.h = (ctx->obs[nd.obs].hi - h.lo) / h.nbins;
    h.slot = gi.slot;
    h.mcol = gi.mcol;
    h.nloc = (int)gi.loc.size();
    for (int l = 0; l < h.nloc; ++l) h.loc2free[l] = ctx->free_pos[gi.loc[l]];
    const int nb = (h.nbins + kThreads1D - 1) / kThreads1D;
    auto alloc = [&](size_t bytes) -> void* {
      void* p = nullptr;
      if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      d.gn_bufs.push_back(p);
      return p;
    };
    Program* sub = static_cast<Program*>(alloc(sizeof(Program)));
    h.partials = static_cast<double*>(alloc(sizeof(double) * (1 + kMaxLocal) * (size_t)nb));
    h.counter = static_cast<unsigned*>(alloc(sizeof(unsigned)));
    GNormDesc* dd = static_cast<GNormDesc*>(alloc(sizeof(GNormDesc)));
    if (!sub || !h.partials || !h.counter || !dd) {
      free_gnorms(d);
      return set_error(ctx, GF_ENOMEM, "device allocation of a grid normalisation failed");
    }
    h.sub = sub;
    CK(cudaMemcpyAsync(sub, &B, sizeof(Program), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(h.counter, 0, sizeof(unsigned), ctx->stream));
    CK(cudaMemcpyAsync(dd, &h, sizeof(GNormDesc), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    d.gn_host[g] = h;
    d.gn_desc[g] = dd;
    d.ngn = (int)g + 1;
  }
  return GF_OK;
}

// Convolution tables and grid normalisations after the normalisation launch (every
// evaluation of a tree with them).
static int enqueue_convs(gf_ctx* ctx, int* launches) {
  DevState& d = ctx->dev;
  for (int c = 0; c < d.nconv; ++c) {
    CK(launch_conv(d.conv_host[c], d.conv_desc[c], weideman(), ctx->prog.nfree, d.derived,
                   ctx->stream));
    if (launches) *launches += 2;
  }
  for (int g = 0; g < d.ngn; ++g) {
    CK(launch_gnorm(d.gn_host[g], d.gn_desc[g], weideman(), ctx->prog.nfree, d.derived,
                    ctx->stream));
    if (launches) *launches += 1;
  }
  return GF_OK;
}

bool has_cycle(gf_ctx* ctx, int id, std::vector<int>& state) {
  if (state[id] == 1) return true;
  if (state[id] == 2) return false;
  state[id] = 1;
  for (int c : ctx->nodes[id].children)
    if (has_cycle(ctx, c, state)) return true;
  state[id] = 2;
  return false;
}

}  // namespace

namespace gfi {

int ensure_compiled(gf_ctx* ctx) {
  if (ctx->compiled) return GF_OK;
  ctx->use_sb = false;
  for (auto& g : ctx->dev.graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  // the serving descriptor holds a copy of the program
  cudaFree(ctx->dev.tick_desc);
  ctx->dev.tick_desc = nullptr;
  ctx->dev.tick_kind = 0;
  if (ctx->root < 0 || !valid_node(ctx, ctx->root))
    return set_error(ctx, GF_ESTATE, "no data set: call gf_set_data first");
  ctx->free_ids.clear();
  ctx->free_pos.assign(ctx->pars.size(), -1);
  for (int i = 0; i < (int)ctx->pars.size(); ++i)
    if (!ctx->pars[i].fixed) {
      ctx->free_pos[i] = (int)ctx->free_ids.size();
      ctx->free_ids.push_back(i);
    }
  const int nf = (int)ctx->free_ids.size();
  std::vector<int> state(ctx->nodes.size(), 0);
  if (has_cycle(ctx, ctx->root, state)) return set_error(ctx, GF_EINVAL, "PDF tree has a cycle");
  const NodeDef& root = ctx->nodes[ctx->root];
  DevState& d = ctx->dev;
  std::vector<int> col_of_obs(ctx->obs.size(), -1);
  for (int k = 0; k < (int)d.obs_ids.size(); ++k) col_of_obs[d.obs_ids[k]] = k;
  ctx->is_tddp = false;
  if (root.type == N_TDDP) {
    if (d.binned || ctx->metric != GF_METRIC_NLL)
      return set_error(ctx, GF_EINVAL, "binned data and binned metrics are for 1D trees");
    if (col_of_obs[root.obs] != 0 || col_of_obs[root.obs2] != 1 || col_of_obs[root.obs3] != 2 ||
        col_of_obs[root.obs4] != 3)
      return set_error(ctx, GF_EINVAL,
                       "time-dependent Dalitz data: columns s12, s13, t, sigma_t in this order");
    if ((int)ctx->pars.size() > 4 * kMaxRes + 8)
      return set_error(ctx, GF_EINVAL, "time-dependent Dalitz: at most 56 parameters in the context");
    ctx->is_tddp = true;
    ctx->is_dalitz = false;
    ctx->has_grid = false;
    TddpPlan& T = ctx->tplan;
    T = TddpPlan{};
    dalitz_geometry(root, T.D);
    T.D.nres = (int)root.res.size();
    T.D.nfree = nf;
    T.nfree = nf;
    T.shape_free = 0;
    for (int r = 0; r < T.D.nres; ++r) {
      const gf_resonance& R = root.res[r];
      DalitzRes& X = T.D.res[r];
      X.channel = R.channel;
      X.spin = R.spin;
      X.p_m0 = R.mass;
      X.p_g0 = R.width;
      X.p_re = R.re;
      X.p_im = R.im;
      X.g_m0 = ctx->free_pos[R.mass];
      X.g_g0 = ctx->free_pos[R.width];
      if (X.g_m0 >= 0 || X.g_g0 >= 0) T.shape_free = 1;
      X.g_re = ctx->free_pos[R.re];
      X.g_im = ctx->free_pos[R.im];
      X.ev_cached = r;
      X.grid_col = r + 1;
    }
    T.p_tau = root.pars[0];
    T.p_x = root.pars[1];
    T.p_y = root.pars[2];
    T.p_s = root.pars[3];
    T.g_tau = ctx->free_pos[T.p_tau];
    T.g_x = ctx->free_pos[T.p_x];
    T.g_y = ctx->free_pos[T.p_y];
    T.g_s = ctx->free_pos[T.p_s];
    T.dens = (root.aux == 1 && root.pars.size() == 7) ? 1 : 0;
    if (T.dens) {
      T.p_b0 = root.pars[4];
      T.p_b1 = root.pars[5];
      T.p_b2 = root.pars[6];
      T.g_b0 = ctx->free_pos[T.p_b0];
      T.g_b1 = ctx->free_pos[T.p_b1];
      T.g_b2 = ctx->free_pos[T.p_b2];
      T.slo = ctx->obs[root.obs4].lo;
      T.shi = ctx->obs[root.obs4].hi;
      const gf_dalitz_kin& K = root.kin;
      T.sc = (K.M * K.M + K.m1 * K.m1 + K.m2 * K.m2 + K.m3 * K.m3) / 3.0;
    } else {
      T.p_b0 = T.p_b1 = T.p_b2 = T.g_b0 = T.g_b1 = T.g_b2 = -1;
    }
    ctx->compiled = true;
    return GF_OK;
  }
  if (root.type == N_DALITZ) {
    if (d.binned || ctx->metric != GF_METRIC_NLL)
      return set_error(ctx, GF_EINVAL, "binned data and binned metrics are for 1D trees");
    ctx->is_dalitz = true;
    DalitzPlan& D = ctx->dplan;
    D = DalitzPlan{};
    dalitz_geometry(root, D);
    if (col_of_obs[root.obs] != 0 || col_of_obs[root.obs2] != 1)
      return set_error(ctx, GF_EINVAL, "Dalitz data set must hold (s12, s13) as columns 0, 1");
    if (nf > 4 * kMaxRes) return set_error(ctx, GF_EINVAL, "too many free parameters");
    D.nres = (int)root.res.size();
    D.nfree = nf;
    int slot = 0;
    for (int r = 0; r < D.nres; ++r) {
      const gf_resonance& R = root.res[r];
      DalitzRes& X = D.res[r];
      X.channel = R.channel;
      X.spin = R.spin;
      X.p_m0 = R.mass;
      X.p_g0 = R.width;
      X.p_re = R.re;
      X.p_im = R.im;
      X.g_m0 = ctx->free_pos[R.mass];
      X.g_g0 = ctx->free_pos[R.width];
      X.g_re = ctx->free_pos[R.re];
      X.g_im = ctx->free_pos[R.im];
      X.ev_cached = (X.g_m0 < 0 && X.g_g0 < 0) ? slot++ : -1;
      X.grid_col = r + 1;
    }
    ctx->has_grid = true;
  } else {
    ctx->is_dalitz = false;
    Program& P = ctx->prog;
    P = Program{};
    P.nobs = (int)d.obs_ids.size();
    if (nf > kMaxFree1D) return set_error(ctx, GF_EINVAL, "1D model: at most 24 free parameters");
    P.nfree = nf;
    Compiler C{ctx, P, col_of_obs};
    std::vector<int> used;
    const int dom = C.walk(ctx->root, used);
    if (dom < 0) return set_error(ctx, GF_EINVAL, C.err);
    if (C.maxdepth > kMaxStack)
      return set_error(ctx, GF_EINVAL, "PDF tree needs a deeper evaluation stack than 4");
    P.root_log = dom;
    int blk = 0;
    ctx->has_grid = false;
    for (int l = 0; l < P.nleaf; ++l) {
      LeafDesc& L = P.leaf[l];
      if (L.nbins > 0) {
        L.grid_first_block = blk;
        L.grid_nblocks = (L.nbins + kThreads - 1) / kThreads;
        blk += L.grid_nblocks;
        ctx->has_grid = true;
      }
    }
    P.ngrid_blocks = blk;
    int rcc = setup_convs(ctx, C.convs);
    if (rcc == GF_OK) rcc = setup_gnorms(ctx, C.gns);
    if (rcc) return rcc;
    if (!C.convs.empty() || !C.gns.empty()) ctx->has_grid = true;  // records from the device
    // the first Voigtian leaf is the one expanded per chunk on sorted data
    P.tay_slot = -1;
    P.tay_obs = 0;
    for (int pc = 0; pc < P.n; ++pc)
      if (P.ins[pc].op == OP_LEAF && P.ins[pc].kind == L_VOIGT) {
        P.tay_slot = P.ins[pc].slot;
        P.tay_obs = P.ins[pc].obs;
        break;
      }
    P.sorted = (d.sorted && P.tay_slot >= 0 && d.sort_obs == P.tay_obs) ? 1 : 0;
    if (ctx->mixture_path) detect_mixture(P);
    else P.mix = 0;
    if (ctx->metric != GF_METRIC_NLL && !d.binned)
      return set_error(ctx, GF_EINVAL, "a binned metric needs a binned data set");
    P.binned = d.binned ? 1 : 0;
    P.metric = ctx->metric;
    P.kbin = d.kbin;
    P.logk = d.kbin > 0 ? std::log(d.kbin) : 0.0;
    P.bw = d.bw;
    P.bs2 = d.bs2;
    if (ctx->mixture_path && !d.binned) detect_logsum(P);
    P.rec_off = 64 * (int)((std::max<size_t>(ctx->pars.size(), 1) + 63) / 64);
    ctx->use_sb = ctx->mixture_path && !d.binned && P.ngrid_blocks > 0 && C.convs.empty() &&
                  C.gns.empty() && detect_sigbkg(P, ctx->sb);
    // the kernels read the program from device memory (it is too large for parameters);
    // stream-ordered copy, then wait: the next launch may go to another stream
    DevState& dv = ctx->dev;
    if (ctx->use_sb && !dv.sbtab)
      CK(cudaMalloc(&dv.sbtab, sizeof(float4) * kSBTabF4 * (size_t)kSBTabCap));
    if (!dv.prog) CK(cudaMalloc(&dv.prog, sizeof(Program)));
    CK(cudaMemcpyAsync(dv.prog, &P, sizeof(Program), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  ctx->compiled = true;
  return GF_OK;
}

}  // namespace gfi

// ---- datasets ----------------------------------------------------------------------------------------------
extern "C" {

int gf_dataset_create(gf_ctx* ctx, int nobs, const int* obs, gf_dataset** ds) {
  if (!ctx || !ds || nobs < 1 || nobs > kMaxObs || !obs) return GF_EINVAL;
  *ds = nullptr;
  for (int k = 0; k < nobs; ++k) {
    if (!valid_obs(ctx, obs[k])) return set_error(ctx, GF_EINVAL, "unknown observable id");
    for (int j = 0; j < k; ++j)
      if (obs[j] == obs[k]) return set_error(ctx, GF_EINVAL, "observable listed twice");
  }
  gf_dataset* d = new (std::nothrow) gf_dataset();
  if (!d) return GF_ENOMEM;
  d->ctx = ctx;
  d->obs.assign(obs, obs + nobs);
  d->cols.resize(nobs);
  *ds = d;
  return GF_OK;
}

int gf_dataset_create_binned(gf_ctx* ctx, int nobs, const int* obs, const int* nbins,
                             const double* counts, const double* errors, gf_dataset** ds) {
  if (!ctx || !ds || !nbins || !counts) return GF_EINVAL;
  *ds = nullptr;
  if (nobs > kMaxObs) return set_error(ctx, GF_EINVAL, "too many observables");
  int64_t nb = 1;
  for (int k = 0; k < nobs; ++k) {
    if (nbins[k] < 1) return set_error(ctx, GF_EINVAL, "nbins must be >= 1");
    nb *= nbins[k];
    if (nb > INT32_MAX) return set_error(ctx, GF_EINVAL, "more than 2^31 bins");
  }
  gf_dataset* d = nullptr;
  int rc = gf_dataset_create(ctx, nobs, obs, &d);
  if (rc) return rc;
  double total = 0.0, vol = 1.0;
  for (int64_t b = 0; b < nb; ++b) {
    if (!(counts[b] >= 0.0) || !std::isfinite(counts[b])) {
      delete d;
      return set_error(ctx, GF_EINVAL, "bin " + std::to_string(b) + ": negative or non-finite count");
    }
    if (errors && !(errors[b] > 0.0 && std::isfinite(errors[b]))) {
      delete d;
      return set_error(ctx, GF_EINVAL, "bin " + std::to_string(b) + ": error must be > 0");
    }
    total += counts[b];
  }
  try {
    for (int k = 0; k < nobs; ++k) {
      const ObsDef& o = ctx->obs[obs[k]];
      vol *= (o.hi - o.lo) / nbins[k];
      d->cols[k].resize(nb);
    }
    d->w.assign(counts, counts + nb);
    d->s2.resize(nb);
    for (int64_t b = 0; b < nb; ++b) {
      d->s2[b] = errors ? errors[b] * errors[b] : std::max(counts[b], 1.0);
      int64_t r = b;
      for (int k = nobs - 1; k >= 0; --k) {  // last observable fastest
        const ObsDef& o = ctx->obs[obs[k]];
        const int64_t i = r % nbins[k];
        r /= nbins[k];
        d->cols[k][b] = o.lo + (o.hi - o.lo) * ((double)i + 0.5) / nbins[k];
      }
    }
  } catch (...) {
    delete d;
    return set_error(ctx, GF_ENOMEM, "host allocation failed");
  }
  d->n = nb;
  d->binned = true;
  d->kbin = total * vol;
  *ds = d;
  return GF_OK;
}

int gf_dataset_add_events(gf_dataset* ds, int64_t n, const double* const* cols) {
  if (!ds || n < 0 || (n > 0 && !cols)) return GF_EINVAL;
  gf_ctx* ctx = ds->ctx;
  if (ds->binned) return set_error(ctx, GF_EINVAL, "a binned data set takes no events");
  for (size_t k = 0; k < ds->obs.size(); ++k) {
    if (n > 0 && !cols[k]) return set_error(ctx, GF_EINVAL, "NULL column");
    const ObsDef& o = ctx->obs[ds->obs[k]];
    for (int64_t i = 0; i < n; ++i) {
      const double v = cols[k][i];
      if (!(v >= o.lo && v <= o.hi))
        return set_error(ctx, GF_EINVAL, "event " + std::to_string(i) + " outside the range of " +
                                             o.name);
    }
  }
  try {
    for (size_t k = 0; k < ds->obs.size(); ++k) ds->cols[k].insert(ds->cols[k].end(), cols[k], cols[k] + n);
  } catch (...) {
    return set_error(ctx, GF_ENOMEM, "host allocation failed");
  }
  ds->n += n;
  return GF_OK;
}

int64_t gf_dataset_size(const gf_dataset* ds) { return ds ? ds->n : -1; }

int gf_dataset_destroy(gf_dataset* ds) {
  delete ds;
  return GF_OK;
}

}  // extern "C"

// ---- device set-up ---------------------------------------------------------------------------------------
static size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

namespace gfi {
size_t device_bytes_for(const gf_ctx* ctx, int root, int64_t n) {
  size_t b = 0;
  const NodeDef& nd = ctx->nodes[root];
  const size_t col = round_up((size_t)std::max<int64_t>(n, 1) * 8, 256);
  if (nd.type == N_DALITZ) {
    const size_t ncell = (size_t)nd.nbx * nd.nby;
    const int nres = (int)nd.res.size();
    b += 2 * col;
    b += ncell + (size_t)(nres + 1) * ncell * 16;
    int ncached = 0;
    for (auto& R : nd.res)
      if (ctx->pars[R.mass].fixed && ctx->pars[R.width].fixed) ++ncached;
    b += (size_t)ncached * n * (ctx->precision == GF_MIXED ? 8 : 16);
    if (ctx->precision == GF_MIXED) b += 3 * (size_t)n * 4;
  } else {
    b += col * 4;  // observables (typically 1-2), or centres + contents + variances
    b += sizeof(float4) * kSBTabF4 * (size_t)kSBTabCap;  // a Voigtian's table of expansions
  }
  return b + (4u << 20);  // work buffers
}
}  // namespace gfi

static int alloc_work(gf_ctx* ctx) {
  DevState& d = ctx->dev;
  const int npar = (int)std::max<size_t>(ctx->pars.size(), 1);
  // theta, then room for the host-computed leaf records of log-sum programs
  const size_t nth = 64 * (size_t)((npar + 63) / 64) + 2 * kLogLeaf * kLeafRec;
  if (!d.theta) CK(cudaMalloc(&d.theta, sizeof(double) * nth));
  if (!d.derived) CK(cudaMalloc(&d.derived, sizeof(double) * (kMaxLeaf * kLeafRec + kMaxCoef)));
  if (!d.counters) {
    CK(cudaMalloc(&d.counters, sizeof(unsigned) * 4));
    CK(cudaMemset(d.counters, 0, sizeof(unsigned) * 4));
  }
  if (!d.norm_out) CK(cudaMalloc(&d.norm_out, sizeof(double) * 64));
  if (!d.h_theta) CK(cudaMallocHost(&d.h_theta, sizeof(double) * nth));
  if (!d.h_result) {
    // NLL and gradient (slots 0 .. nfree) and the data-check flag (slot 63) are written by
    // the kernels straight into this pinned buffer through its device mapping: no copy
    // back per evaluation
    CK(cudaMallocHost(&d.h_result, sizeof(double) * 64));
    std::memset(d.h_result, 0, sizeof(double) * 64);
    void* p = nullptr;
    CK(cudaHostGetDevicePointer(&p, d.h_result, 0));
    d.result = static_cast<double*>(p);
    d.flag = reinterpret_cast<int*>(d.result + 63);
  }
  if (!d.ev0) CK(cudaEventCreate(&d.ev0));
  if (!d.ev1) CK(cudaEventCreate(&d.ev1));
  if (!d.evm) CK(cudaEventCreate(&d.evm));
  return GF_OK;
}

static int grow(gf_ctx* ctx, double** p, size_t* cap, size_t need) {
  if (*cap >= need) return GF_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  CK(cudaMalloc(p, need * sizeof(double)));
  *cap = need;
  return GF_OK;
}

// Shared tail of gf_set_data / gf_set_data_device once the columns are on the device.
static int finish_set_data(gf_ctx* ctx) {
  DevState& d = ctx->dev;
  int rc = alloc_work(ctx);
  if (rc) return rc;
  rc = ensure_compiled(ctx);
  if (rc) return rc;
  if (ctx->is_tddp) {
    const TddpPlan& T = ctx->tplan;
    // every block resident, events split evenly over them (>= 64 per block)
    const int64_t want = (d.n + 63) / 64;
    d.nblocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(want, (int64_t)ctx->sm_count * kTddpBlocksPerSm));
    rc = grow(ctx, &d.partials, &d.partials_cap, (size_t)std::max(d.nblocks, 2048) * 64);
    if (rc) return rc;
    const size_t ncell = (size_t)T.D.nbx * T.D.nby;
    cudaFree(d.inside);
    cudaFree(d.tddp_cache);
    cudaFree(d.tddp_gcols);
    cudaFree(d.tddp_gram);
    d.inside = nullptr;
    d.tddp_cache = nullptr;
    d.tddp_gcols = d.tddp_gram = nullptr;
    CK(cudaMalloc(&d.inside, ncell));
    CK(cudaMalloc(&d.tddp_cache, sizeof(float4) * 2 * std::max(T.D.nres, 1) * (size_t)std::max<int64_t>(d.n, 1)));
    CK(cudaMalloc(&d.tddp_gcols, sizeof(double2) * 2 * std::max(T.D.nres, 1) * ncell));
    CK(cudaMalloc(&d.tddp_gram, sizeof(double2) * 3 * (kMaxRes + 1) * (kMaxRes + 1)));
    cudaFree(d.tddp_dcache);
    cudaFree(d.tddp_normd);
    d.tddp_dcache = nullptr;
    d.tddp_normd = nullptr;
    // N and dN/dtheta: from the direct cell pass (free shapes) or published by the event
    // pass's first block to finish (fixed shapes)
    CK(cudaMalloc(&d.tddp_normd, sizeof(double) * 64));
    if (T.shape_free) {
      CK(cudaMalloc(&d.tddp_dcache, sizeof(float4) * 4 * std::max(T.D.nres, 1) *
                                        (size_t)std::max<int64_t>(d.n, 1)));
      rc = grow(ctx, &d.partials2, &d.partials2_cap, (size_t)4096 * 64);
      if (rc) return rc;
    }
    d.tddp_shape.clear();
    d.tddp_ready = false;
    return GF_OK;
  }
  // event-stream grid: a multiple of the SM count, capped by the work
  int per_sm;
  if (ctx->is_dalitz) {
    bool co = ctx->dplan.nres > 0;
    for (int r = 0; r < ctx->dplan.nres; ++r) co = co && ctx->dplan.res[r].ev_cached >= 0;
    per_sm = dalitz_blocks_per_sm(ctx->precision == GF_MIXED, true, co, ctx->dplan.nfree);
  } else if (ctx->prog.logsum) {
    per_sm = events_logsum_blocks_per_sm(ctx->prog);
  } else if (ctx->use_sb) {
    per_sm = sigbkg_blocks_per_sm(false);
  } else {
    per_sm = events_1d_blocks_per_sm(true, events_1d_smem(ctx->prog, true, kThreads1D),
                                     ctx->prog.mix > 0);
  }
  per_sm = std::max(1, std::min(per_sm, 8));
  // signal + background form: 16 events per thread at least, so that sorted data reach the
  // expanded (chunked) event loop at every size
  const int64_t items = ctx->is_dalitz ? d.n : ctx->use_sb ? (d.n + 15) / 16 : (d.n + 1) / 2;
  const int tpb = ctx->is_dalitz ? kThreads : ctx->use_sb ? sigbkg_threads(false) : kThreads1D;
  const int64_t want = (items + tpb - 1) / tpb;
  d.nblocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)ctx->sm_count * per_sm));
  d.nblocks_mixed = d.nblocks;
  if (ctx->use_sb) {  // the mixed plan: its own block size and resident blocks per SM
    const int pm = std::max(1, std::min(sigbkg_blocks_per_sm(true), 8));
    const int tm = sigbkg_threads(true);
    d.nblocks_mixed = (int)std::max<int64_t>(
        1, std::min<int64_t>((items + tm - 1) / tm, (int64_t)ctx->sm_count * pm));
  }
  rc = grow(ctx, &d.partials, &d.partials_cap,
            (size_t)std::max(std::max(d.nblocks, d.nblocks_mixed), 2048) * 64);
  if (rc) return rc;
  // norm-side partials: 1D grid blocks x 4, Gram chunks x groups x 16, cell blocks x 49
  size_t need2 = (size_t)4096 * 64;
  if (!ctx->is_dalitz) need2 = std::max(need2, (size_t)ctx->prog.ngrid_blocks * 4 + 64);
  rc = grow(ctx, &d.partials2, &d.partials2_cap, need2);
  if (rc) return rc;
  if (ctx->is_dalitz) {
    const DalitzPlan& D = ctx->dplan;
    const size_t ncell = (size_t)D.nbx * D.nby;
    cudaFree(d.inside);
    cudaFree(d.grid_cols);
    cudaFree(d.gram);
    cudaFree(d.ev_cache);
    cudaFree(d.fcols);
    cudaFree(d.todo);
    d.inside = nullptr; d.grid_cols = nullptr; d.gram = nullptr; d.ev_cache = nullptr;
    d.fcols = nullptr; d.todo = nullptr;
    CK(cudaMalloc(&d.inside, ncell));
    CK(cudaMalloc(&d.grid_cols, (size_t)(D.nres + 1) * ncell * 16));
    CK(cudaMalloc(&d.gram, sizeof(double) * 2 * (kMaxRes + 1) * (kMaxRes + 1)));
    CK(cudaMalloc(&d.todo, sizeof(int) * kMaxRes));
    int ncached = 0;
    for (int r = 0; r < D.nres; ++r) ncached += D.res[r].ev_cached >= 0 ? 1 : 0;
    const bool mixed = ctx->precision == GF_MIXED;
    if (ncached > 0 && d.n > 0)
      CK(cudaMalloc(&d.ev_cache, (size_t)ncached * d.n * (mixed ? 8 : 16)));
    if (mixed && d.n > 0) {
      CK(cudaMalloc(&d.fcols, 3 * (size_t)d.n * sizeof(float)));
      CK(launch_dalitz_fcols(D, d.cols[0], d.cols[1], d.n, d.fcols, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    }
    d.ev_m0.assign(D.nres, NAN);
    d.ev_g0.assign(D.nres, NAN);
    d.col_m0.assign(D.nres, NAN);
    d.col_g0.assign(D.nres, NAN);
    d.gram_valid = false;
    d.mask_built = false;
  }
  return GF_OK;
}

// ---- sorted layout of owned 1D columns (k_sort.cu) ------------------------------------
// Worth it when the chunked event loop will run: a Voigtian leaf, columns the context
// owns (the caller's device columns are never reordered) and at least kChunk/2 events
// per thread of the event launch.
static bool sort_eligible(const gf_ctx* ctx) {
  const DevState& d = ctx->dev;
  return ctx->event_sort && ctx->compiled && !ctx->is_dalitz && !ctx->is_tddp && d.owns_cols &&
         !d.binned &&
         ctx->prog.tay_slot >= 0 && d.n < INT32_MAX &&
         d.n >= (int64_t)(kChunk / 2) * d.nblocks * kThreads1D;
}

// Reorder the columns ascending by the Voigtian's observable and keep the permutation.
// A pure optimisation: if scratch memory is short the data stay as they are.
static int sort_events(gf_ctx* ctx) {
  DevState& d = ctx->dev;
  const int64_t n = d.n;
  const int ov = ctx->prog.tay_obs;
  cudaStream_t st = ctx->stream;
  const size_t bytes = round_up((size_t)std::max<int64_t>(n + 2, 2) * 8, 256);
  size_t tb = 0;
  CK(sort_by_key_f64(d.cols[ov], nullptr, nullptr, nullptr, n, nullptr, &tb, st));
  std::vector<double*> fresh(d.nobs, nullptr);
  int32_t* ptmp = nullptr;
  int32_t* pout = d.perm;
  void* temp = nullptr;
  bool ok = cudaMalloc(&ptmp, sizeof(int32_t) * n) == cudaSuccess &&
            (pout || cudaMalloc(&pout, sizeof(int32_t) * n) == cudaSuccess) &&
            cudaMalloc(&temp, std::max<size_t>(tb, 16)) == cudaSuccess;
  for (int k = 0; ok && k < d.nobs; ++k)
    ok = cudaMalloc(&fresh[k], bytes) == cudaSuccess &&
         cudaMemsetAsync(fresh[k], 0, bytes, st) == cudaSuccess;
  if (ok) ok = sort_by_key_f64(d.cols[ov], fresh[ov], ptmp, pout, n, temp, &tb, st) == cudaSuccess;
  for (int k = 0; ok && k < d.nobs; ++k)
    if (k != ov) ok = launch_gather(d.cols[k], pout, fresh[k], n, st) == cudaSuccess;
  if (ok) ok = cudaStreamSynchronize(st) == cudaSuccess;
  cudaFree(ptmp);
  cudaFree(temp);
  if (!ok) {
    cudaGetLastError();
    for (double* p : fresh) cudaFree(p);
    if (pout != d.perm) cudaFree(pout);
    return GF_OK;
  }
  for (int k = 0; k < d.nobs; ++k) {
    cudaFree(d.cols[k]);
    d.cols[k] = fresh[k];
  }
  d.perm = pout;
  d.sorted = true;
  d.sort_obs = ov;
  // kernels read the sorted flag from the program; captured graphs and the serving
  // descriptor hold the old column pointers
  ctx->prog.sorted = 1;
  CK(cudaMemcpyAsync(d.prog, &ctx->prog, sizeof(Program), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  for (auto& g : d.graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  cudaFree(d.tick_desc);
  d.tick_desc = nullptr;
  d.tick_kind = 0;
  return GF_OK;
}

// The columns were overwritten in the caller's order: back to the strided event loop.
static int mark_unsorted(gf_ctx* ctx) {
  DevState& d = ctx->dev;
  d.evals_since_load = 0;
  if (!d.sorted) return GF_OK;
  d.sorted = false;
  d.sort_obs = -1;
  if (ctx->compiled && !ctx->is_dalitz && !ctx->is_tddp) {
    ctx->prog.sorted = 0;
    CK(cudaMemcpyAsync(d.prog, &ctx->prog, sizeof(Program), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return GF_OK;
}

extern "C" int gf_set_data(gf_ctx* ctx, int root, const gf_dataset* ds) {
  if (!ctx || !ds || ds->ctx != ctx || !valid_node(ctx, root)) return GF_EINVAL;
  if (ctx->eval_in_flight)
    return set_error(ctx, GF_ESTATE, "an evaluation started by gf_nll_grad_start is not finished");
  CK(cudaSetDevice(ctx->device));
  const NodeDef& nd = ctx->nodes[root];
  if (nd.type == N_DALITZ || nd.type == N_TDDP) {
    // both observables as columns 0, 1 and every event inside the kinematic region
    if (ds->obs.size() < 2 || ds->obs[0] != nd.obs || ds->obs[1] != nd.obs2)
      return set_error(ctx, GF_EINVAL, "Dalitz data set must hold (s12, s13) as columns 0, 1");
    if (nd.type == N_TDDP) {
      if (ds->obs.size() != 4 || ds->obs[2] != nd.obs3 || ds->obs[3] != nd.obs4)
        return set_error(ctx, GF_EINVAL,
                         "time-dependent Dalitz data: columns s12, s13, t, sigma_t in this order");
      for (int64_t i = 0; i < ds->n; ++i)
        if (!(ds->cols[3][i] > 0.0))
          return set_error(ctx, GF_EINVAL, "event " + std::to_string(i) + ": sigma_t must be > 0");
    }
    DalitzPlan D{};
    dalitz_geometry(nd, D);
    for (int64_t i = 0; i < ds->n; ++i)
      if (!dalitz_inside_host(D, ds->cols[0][i], ds->cols[1][i]))
        return set_error(ctx, GF_EINVAL,
                         "event " + std::to_string(i) + " outside the Dalitz kinematic region");
  }
  cudaStreamSynchronize(ctx->stream);
  free_dev(ctx);
  DevState& d = ctx->dev;
  d.nobs = (int)ds->obs.size();
  d.n = ds->n;
  d.obs_ids = ds->obs;
  d.owns_cols = true;
  const size_t bytes = round_up((size_t)std::max<int64_t>(ds->n + 2, 2) * 8, 256);
  for (int k = 0; k < d.nobs; ++k) {
    double* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      free_dev(ctx);
      return set_error(ctx, GF_ENOMEM, "device allocation of the event columns failed");
    }
    d.cols.push_back(p);
    CK(cudaMemsetAsync(p, 0, bytes, ctx->stream));
    if (ds->n > 0)
      CK(cudaMemcpyAsync(p, ds->cols[k].data(), 8 * ds->n, cudaMemcpyHostToDevice, ctx->stream));
  }
  if (ds->binned) {
    d.binned = true;
    d.kbin = ds->kbin;
    for (double** dst : {&d.bw, &d.bs2}) {
      if (cudaMalloc(dst, bytes) != cudaSuccess) {
        cudaGetLastError();
        free_dev(ctx);
        return set_error(ctx, GF_ENOMEM, "device allocation of the bin contents failed");
      }
      CK(cudaMemsetAsync(*dst, 0, bytes, ctx->stream));
    }
    if (ds->n > 0) {
      CK(cudaMemcpyAsync(d.bw, ds->w.data(), 8 * ds->n, cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemcpyAsync(d.bs2, ds->s2.data(), 8 * ds->n, cudaMemcpyHostToDevice, ctx->stream));
    }
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->root = root;
  ctx->compiled = false;
  int rc = finish_set_data(ctx);
  if (rc == GF_OK && sort_eligible(ctx)) rc = sort_events(ctx);
  return rc;
}

extern "C" int gf_set_data_device(gf_ctx* ctx, int root, int nobs, const int* obs, int64_t n,
                                  const double* const* dev_cols) {
  if (!ctx || !valid_node(ctx, root) || nobs < 1 || nobs > kMaxObs || !obs || n < 0 ||
      !dev_cols)
    return GF_EINVAL;
  if (ctx->eval_in_flight)
    return set_error(ctx, GF_ESTATE, "an evaluation started by gf_nll_grad_start is not finished");
  for (int k = 0; k < nobs; ++k) {
    if (!valid_obs(ctx, obs[k]) || !dev_cols[k]) return GF_EINVAL;
    if (reinterpret_cast<uintptr_t>(dev_cols[k]) % 16 != 0)
      return set_error(ctx, GF_EINVAL, "device columns must be 16-byte aligned");
  }
  CK(cudaSetDevice(ctx->device));
  cudaStreamSynchronize(ctx->stream);
  free_dev(ctx);
  DevState& d = ctx->dev;
  d.nobs = nobs;
  d.n = n;
  d.obs_ids.assign(obs, obs + nobs);
  d.owns_cols = false;
  for (int k = 0; k < nobs; ++k) d.cols.push_back(const_cast<double*>(dev_cols[k]));
  ctx->root = root;
  ctx->compiled = false;
  return finish_set_data(ctx);
}

// ---- evaluation ----------------------------------------------------------------------------------------------
// The device copy of this evaluation's table layout (uploaded with theta).
static const SBTabHdr* sbtab_hdr(gf_ctx* ctx) {
  return reinterpret_cast<const SBTabHdr*>(ctx->dev.theta + ctx->prog.rec_off);
}
// Blocks of the normalisation launch that build the table: the SMs the grids leave, at
// least 64 (16 k threads: one entry each for most lines)
static int sbtab_blocks(const gf_ctx* ctx) {
  return std::max(64, ctx->sm_count - ctx->prog.ngrid_blocks);
}

static int fill_theta_host(gf_ctx* ctx, const double* theta) {
  DevState& d = ctx->dev;
  // the queued evaluation's graph reads the pinned theta when the stream reaches it
  if (ctx->eval_in_flight)
    return set_error(ctx, GF_ESTATE, "an evaluation started by gf_nll_grad_start is not finished");
  const int np = (int)ctx->pars.size();
  for (int i = 0; i < np; ++i) d.h_theta[i] = ctx->pars[i].value;
  for (size_t k = 0; k < ctx->free_ids.size(); ++k) {
    if (!std::isfinite(theta[k])) return set_error(ctx, GF_EINVAL, "non-finite theta");
    d.h_theta[ctx->free_ids[k]] = theta[k];
  }
  sbtab_fill(ctx, d.h_theta);
  if (ctx->compiled && ctx->prog.logsum) {
    // the log-sum kernel's leaf records (analytic leaves: leafrec.h), here once instead of
    // in FP64 in every block; doubles, then float pairs (hi rounded, lo the rest rounded)
    const Program& P = ctx->prog;
    double* rec = d.h_theta + P.rec_off;
    float* pf = reinterpret_cast<float*>(rec + kLogLeaf * kLeafRec);
    for (int l = 0; l < P.nleaf; ++l) {
      double* r = rec + l * kLeafRec;
      for (int k = 0; k < kLeafRec; ++k) r[k] = 0.0;
      analytic_leaf_record(P.leaf[l], d.h_theta, (P.leaf[l].aux & kRawLeaf) != 0, r);
      for (int k = 0; k < kLeafRec; ++k) {
        const float hi = (float)r[k];
        pf[2 * (l * kLeafRec + k)] = hi;
        pf[2 * (l * kLeafRec + k) + 1] = (float)(r[k] - (double)hi);
      }
    }
  }
  return GF_OK;
}

// Queue the upload of theta on the context's stream.
static int enqueue_uploads(gf_ctx* ctx) {
  DevState& d = ctx->dev;
  int np = (int)ctx->pars.size();
  if (ctx->compiled && ctx->prog.logsum)
    np = ctx->prog.rec_off + 2 * kLogLeaf * kLeafRec;  // with the leaf records
  else
    np = theta_all_size(ctx);  // with the table's layout (signal + background form)
  if (np > 0)
    CK(cudaMemcpyAsync(d.theta, d.h_theta, sizeof(double) * np, cudaMemcpyHostToDevice,
                       ctx->stream));
  return GF_OK;
}

static int upload_theta(gf_ctx* ctx, const double* theta) {
  int rc = fill_theta_host(ctx, theta);
  if (rc) return rc;
  return enqueue_uploads(ctx);
}

// Dalitz: true when no cache needs (re)building for this evaluation (mask, per-event and
// grid columns of fixed-shape resonances, Gram matrix); *direct: free shapes present.
static bool dalitz_is_steady(gf_ctx* ctx, bool mixed, bool* direct) {
  DevState& d = ctx->dev;
  const DalitzPlan& D = ctx->dplan;
  const bool second = ctx->precision == GF_MIXED && !mixed;
  const std::vector<double>& cm0 = second ? d.ev64_m0 : d.ev_m0;
  const std::vector<double>& cg0 = second ? d.ev64_g0 : d.ev_g0;
  *direct = false;
  if (!d.mask_built || cm0.size() != (size_t)D.nres || d.col_m0.size() != (size_t)D.nres)
    return false;
  int ncached = 0;
  for (int r = 0; r < D.nres; ++r) {
    const DalitzRes& R = D.res[r];
    const double m0 = d.h_theta[R.p_m0], g0 = d.h_theta[R.p_g0];
    if (R.ev_cached >= 0) {
      ++ncached;
      if (!(cm0[r] == m0 && cg0[r] == g0) || !(d.col_m0[r] == m0 && d.col_g0[r] == g0))
        return false;
    } else {
      *direct = true;
    }
  }
  if (second && ncached > 0 && !d.ev_cache64) return false;
  return *direct || d.gram_valid;
}

static DalitzBufs dalitz_bufs(gf_ctx* ctx, double* out_logp, bool mixed = true) {
  DevState& d = ctx->dev;
  DalitzBufs B{};
  B.s12 = d.cols[0];
  B.s13 = d.cols[1];
  B.sf = d.fcols;
  B.n = d.n;
  B.ev_cache = (ctx->precision == GF_MIXED && !mixed) ? d.ev_cache64 : d.ev_cache;
  B.grid_cols = d.grid_cols;
  B.inside = d.inside;
  B.gram = d.gram;
  B.norm_out = d.norm_out;
  B.partials = d.partials;
  B.partials2 = d.partials2;
  B.counter = d.counters;
  B.counter2 = d.counters + 1;
  B.result = d.result;
  B.out_logp = out_logp;
  return B;
}

// Dalitz caches: rebuild event / grid columns of fixed-shape resonances whose (m0,
// Gamma0) differ from those the caches hold; decide the normalisation mode.
static int dalitz_prepare(gf_ctx* ctx, int* norm_mode, int* launches, bool mixed) {
  if (!ctx->is_dalitz) return set_error(ctx, GF_ESTATE, "dalitz_prepare on a 1D context");
  DevState& d = ctx->dev;
  const DalitzPlan& D = ctx->dplan;
  // the per-event cache matching the arithmetic of this evaluation: FP32 pairs for
  // mixed evaluations, FP64 pairs otherwise (a mixed context keeps a second, FP64 cache
  // for the refinement stage of its fits)
  const bool second = ctx->precision == GF_MIXED && !mixed;
  void*& cache = second ? d.ev_cache64 : d.ev_cache;
  std::vector<double>& cm0 = second ? d.ev64_m0 : d.ev_m0;
  std::vector<double>& cg0 = second ? d.ev64_g0 : d.ev_g0;
  if (cm0.size() != (size_t)D.nres) {
    cm0.assign(D.nres, NAN);
    cg0.assign(D.nres, NAN);
  }
  int ncached = 0;
  for (int r = 0; r < D.nres; ++r) ncached += D.res[r].ev_cached >= 0 ? 1 : 0;
  if (second && !cache && ncached > 0 && d.n > 0)
    CK(cudaMalloc(&cache, (size_t)ncached * d.n * 16));
  if (!d.mask_built) {
    CK(launch_dalitz_mask(D, d.inside, ctx->stream));
    (*launches)++;
    d.mask_built = true;
  }
  bool ev_stale = false;
  std::vector<int> todo;
  bool any_free_shape = false;
  for (int r = 0; r < D.nres; ++r) {
    const DalitzRes& R = D.res[r];
    const double m0 = d.h_theta[R.p_m0], g0 = d.h_theta[R.p_g0];
    if (R.ev_cached >= 0) {
      if (!(cm0[r] == m0 && cg0[r] == g0)) ev_stale = true;
      if (!(d.col_m0[r] == m0 && d.col_g0[r] == g0)) todo.push_back(r);
    } else {
      any_free_shape = true;
    }
  }
  if (ev_stale && d.n > 0) {
    CK(launch_dalitz_ev_cache(D, mixed, d.theta, d.cols[0], d.cols[1], d.n, cache, ctx->stream));
    (*launches)++;
  }
  for (int r = 0; r < D.nres; ++r)
    if (D.res[r].ev_cached >= 0) {
      cm0[r] = d.h_theta[D.res[r].p_m0];
      cg0[r] = d.h_theta[D.res[r].p_g0];
    }
  if (!todo.empty()) {
    CK(cudaMemcpyAsync(d.todo, todo.data(), sizeof(int) * todo.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(launch_dalitz_grid_cols(D, d.theta, d.todo, (int)todo.size(), d.grid_cols, d.inside,
                               ctx->stream));
    (*launches)++;
    for (int r : todo) {
      d.col_m0[r] = d.h_theta[D.res[r].p_m0];
      d.col_g0[r] = d.h_theta[D.res[r].p_g0];
    }
    d.gram_valid = false;
    // the todo buffer is read by the kernel: keep the host vector alive until then
    CK(cudaStreamSynchronize(ctx->stream));
  }
  if (!any_free_shape) {
    if (!d.gram_valid) {
      DalitzBufs B = dalitz_bufs(ctx, nullptr);
      CK(launch_dalitz_gram(D, B, ctx->stream));
      (*launches)++;
      d.gram_valid = true;
    }
    *norm_mode = DN_GRAM;
  } else {
    *norm_mode = DN_DIRECT;
  }
  return GF_OK;
}

namespace gfi {

// The evaluation after any cache maintenance: the normalisation and event kernels, the
// result and data-check downloads, timing events.  capturing: the stream is being
// captured into a graph, which then also holds the theta upload from the pinned buffer.
static int enqueue_steady(gf_ctx* ctx, bool grad, bool fp64, int mode, bool capturing,
                          int* launches) {
  DevState& d = ctx->dev;
  // Timing events: inside a stream capture a plain record only orders the capture and
  // never records the event, so there they become external event-record nodes.
  const unsigned evf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  const bool with_upload = capturing;
  const int nf = (int)ctx->free_ids.size();
  if (with_upload) {
    const int rc = enqueue_uploads(ctx);
    if (rc) return rc;
  }
  CK(cudaEventRecordWithFlags(d.ev0, ctx->stream, evf));
  if (ctx->is_dalitz) {
    const bool mixed = ctx->precision == GF_MIXED && !fp64;
    DalitzBufs B = dalitz_bufs(ctx, nullptr, mixed);
    if (mode == DN_DIRECT) {
      const int ncell_blocks = (int)std::min<int64_t>(
          ((int64_t)ctx->dplan.nbx * ctx->dplan.nby + kThreads - 1) / kThreads,
          (int64_t)ctx->sm_count);  // a few cells per thread: amortise the block set-up
      // the normalisation integral and its gradient in FP64 in every mode
      CK(launch_dalitz_norm_direct(ctx->dplan, false, grad, d.theta, B, ncell_blocks,
                                   ctx->stream));
      (*launches)++;
    }
    CK(cudaEventRecordWithFlags(d.evm, ctx->stream, evf));
    CK(launch_dalitz_events(ctx->dplan, mixed, grad, false, mode, d.theta, B, d.nblocks,
                            ctx->stream));
    (*launches)++;
  } else {
    const WeidCoef& W = weideman();
    if (ctx->has_grid) {
      const bool tab = ctx->use_sb && d.sbtab;
      CK(launch_norm_1d(ctx->prog, d.prog, W, d.theta, d.partials2, d.counters + 1, d.derived,
                        tab ? sbtab_hdr(ctx) : nullptr, tab ? d.sbtab : nullptr,
                        sbtab_blocks(ctx), ctx->stream));
      (*launches)++;
      const int rc = enqueue_convs(ctx, launches);
      if (rc) return rc;
    }
    Cols cols{};
    for (int k = 0; k < d.nobs; ++k) cols.c[k] = d.cols[k];
    CK(cudaEventRecordWithFlags(d.evm, ctx->stream, evf));
    if (ctx->use_sb) {
      const bool mixed = ctx->precision == GF_MIXED && !fp64;
      CK(launch_sigbkg(ctx->sb, W, d.prog, d.cols[ctx->prog.ins[ctx->prog.mix_leaf[0]].obs], d.n,
                       d.derived, d.partials, d.counters, d.result, nullptr, nullptr, grad, mixed,
                       mixed ? d.nblocks_mixed : d.nblocks, sbtab_hdr(ctx), d.sbtab,
                       ctx->stream));
    } else {
      CK(launch_events_1d(ctx->prog, d.prog, W, cols, d.n, d.theta, d.derived, d.partials,
                          d.counters, d.result, nullptr, nullptr, grad, false,
                          ctx->has_grid ? 0 : 1, d.nblocks, ctx->stream));
    }
    (*launches)++;
  }
  CK(cudaEventRecordWithFlags(d.ev1, ctx->stream, evf));
  (void)nf;  // the result and the data-check flag are already in d.h_result (mapped)
  return GF_OK;
}

// Time-dependent Dalitz model: theta upload, the caches on the first evaluation after a
// data load (cell mask, per-event amplitudes, grid sums; the resonance shapes are fixed),
// then the event pass (every block forms N from the grid sums), storing per-event log P
// when out_logp is given; launched directly (no graph).
static int tddp_enqueue(gf_ctx* ctx, bool grad, double* out_logp, int* launches) {
  DevState& d = ctx->dev;
  const TddpPlan& T = ctx->tplan;
  int rc = enqueue_uploads(ctx);
  if (rc) return rc;
  CK(cudaEventRecord(d.ev0, ctx->stream));
  if (!T.shape_free) {
    if (!d.tddp_ready) {
      CK(launch_dalitz_mask(T.D, d.inside, ctx->stream));
      CK(launch_tddp_cache(T, d.theta, d.cols[0], d.cols[1], d.n, d.tddp_cache, ctx->stream));
      CK(launch_tddp_gram(T, d.theta, d.inside, d.tddp_gcols, d.tddp_gram, ctx->stream));
      *launches += 4;
      d.tddp_ready = true;
    }
  } else {
    // free shapes: the per-event amplitudes and their derivatives whenever a mass or
    // width changed, and N with its gradient by a direct cell pass at every evaluation
    std::vector<double> shape;
    for (int r = 0; r < T.D.nres; ++r) {
      shape.push_back(d.h_theta[T.D.res[r].p_m0]);
      shape.push_back(d.h_theta[T.D.res[r].p_g0]);
    }
    if (!d.tddp_ready) {
      CK(launch_dalitz_mask(T.D, d.inside, ctx->stream));
      (*launches)++;
    }
    if (!d.tddp_ready || shape != d.tddp_shape) {
      CK(launch_tddp_cache_free(T, d.theta, d.cols[0], d.cols[1], d.n, d.tddp_cache,
                                d.tddp_dcache, ctx->stream));
      (*launches)++;
      d.tddp_shape = shape;
      d.tddp_ready = true;
    }
    const int64_t ncell = (int64_t)T.D.nbx * T.D.nby;
    const int nb = (int)std::max<int64_t>(
        1, std::min<int64_t>((ncell + kThreads - 1) / kThreads, (int64_t)ctx->sm_count * 2));
    CK(launch_tddp_norm_direct(T, d.theta, d.inside, d.partials2, d.counters + 1, d.tddp_normd,
                               nb, ctx->stream));
    (*launches)++;
  }
  CK(cudaEventRecord(d.evm, ctx->stream));
  const double* cols[4] = {d.cols[0], d.cols[1], d.cols[2], d.cols[3]};
  CK(launch_tddp_events(T, grad, d.theta, cols, d.n, d.tddp_cache, d.tddp_dcache, d.tddp_gram,
                        T.shape_free ? d.tddp_normd : nullptr, d.tddp_normd, d.partials,
                        d.counters,
                        d.result, out_logp, d.nblocks, weideman(), ctx->stream));
  (*launches)++;
  CK(cudaEventRecord(d.ev1, ctx->stream));
  return GF_OK;  // result and data-check flag: written into d.h_result (mapped)
}

int evaluate_async(gf_ctx* ctx, const double* theta, bool grad, bool fp64) {
  int rc = ensure_compiled(ctx);
  if (rc) return rc;
  DevState& d = ctx->dev;
  if (!d.theta) return set_error(ctx, GF_ESTATE, "no data set");
  CK(cudaSetDevice(ctx->device));
  rc = fill_theta_host(ctx, theta);
  if (rc) return rc;
  if (ctx->is_tddp) {
    int launches = 0;
    rc = tddp_enqueue(ctx, grad, nullptr, &launches);
    ctx->last_launches = launches;
    ctx->last_graph = false;
    return rc;
  }
  // steady state: replay the evaluation graph of this (grad, fp64, normalisation mode)
  bool direct = false;
  const bool mixed = ctx->precision == GF_MIXED && !fp64;
  const bool steady = !ctx->is_dalitz || dalitz_is_steady(ctx, mixed, &direct);
  if (steady && ctx->graphs && !d.graph_off) {
    const int key = (grad ? 1 : 0) | (fp64 ? 2 : 0) | (direct ? 4 : 0) | (d.cur_set << 3);
    int launches = 0;
    if (!d.graph[key]) {
      // capture once; if the capture or instantiation fails for any reason the context
      // stops using graphs and this and later evaluations launch directly
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      const std::string err_before = ctx->err;
      std::string why;
      cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        why = std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e);
      } else {
        const int rc_cap =
            enqueue_steady(ctx, grad, fp64, direct ? DN_DIRECT : DN_GRAM, true, &launches);
        e = cudaStreamEndCapture(ctx->stream, &g);
        if (rc_cap != GF_OK) why = ctx->err;
        else if (e != cudaSuccess || !g)
          why = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e);
        else if ((e = cudaGraphInstantiate(&ge, g, 0)) != cudaSuccess)
          why = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
      }
      if (g) cudaGraphDestroy(g);
      if (!why.empty()) {
        if (ge) cudaGraphExecDestroy(ge);
        cudaGetLastError();
        ctx->err = err_before;
        d.graph_off = true;
        d.graph_why = why;
        launches = 0;
      } else {
        d.graph[key] = ge;
      }
    } else {
      launches = (ctx->is_dalitz ? (direct ? 2 : 1)
                                 : (ctx->has_grid ? 2 + 2 * d.nconv + d.ngn : 1));
    }
    if (!d.graph_off) {
      CK(cudaGraphLaunch(d.graph[key], ctx->stream));
      ctx->last_launches = launches;
      ctx->last_graph = true;
      return GF_OK;
    }
  }
  ctx->last_graph = false;
  // cache maintenance first (Dalitz), then the evaluation
  rc = enqueue_uploads(ctx);
  if (rc) return rc;
  int launches = 0, mode = DN_GRAM;
  if (ctx->is_dalitz) {
    rc = dalitz_prepare(ctx, &mode, &launches, mixed);
    if (rc) return rc;
  }
  rc = enqueue_steady(ctx, grad, fp64, mode, false, &launches);
  if (rc) return rc;
  ctx->last_launches = launches;
  return GF_OK;
}

int evaluate_finish(gf_ctx* ctx, double* nll, double* grad, bool grad_wanted) {
  DevState& d = ctx->dev;
  CK(cudaStreamSynchronize(ctx->stream));
  float ms = 0.f;
  // timings are informative: a failure makes them NaN and must not linger as the
  // runtime's last error (the next launch check would report it)
  ctx->last_ms = ctx->last_stream_ms = NAN;
  if (cudaEventElapsedTime(&ms, d.ev0, d.ev1) == cudaSuccess) ctx->last_ms = ms;
  else cudaGetLastError();
  if (cudaEventElapsedTime(&ms, d.evm, d.ev1) == cudaSuccess) ctx->last_stream_ms = ms;
  else cudaGetLastError();
  const int bad = *reinterpret_cast<const int*>(d.h_result + 63);
  if (bad) {
    *reinterpret_cast<volatile int*>(d.h_result + 63) = 0;
    *nll = INFINITY;
    return set_error(ctx, GF_EINVAL, "gf_update_data: an event lies outside its range/region");
  }
  const int nf = (int)ctx->free_ids.size();
  double v = d.h_result[0];
  bool finite = std::isfinite(v);
  if (grad_wanted && grad)
    for (int k = 0; k < nf; ++k) {
      grad[k] = d.h_result[1 + k];
      finite = finite && std::isfinite(grad[k]);
    }
  if (!finite) {
    *nll = INFINITY;
    return set_error(ctx, GF_ENONFINITE, "non-finite likelihood: some P_i <= 0 or not finite");
  }
  *nll = v;
  return GF_OK;
}

void sbtab_fill(const gf_ctx* ctx, double* theta_all) {
  if (!ctx->compiled || !ctx->use_sb) return;
  const Program& P = ctx->prog;
  const DevState& d = ctx->dev;
  SBTabHdr H{};
  // sorted events with at least 8 per thread of both plans' launches go in chunks that
  // expand w themselves: no table then
  const int64_t t_max = std::max<int64_t>((int64_t)d.nblocks * sigbkg_threads(false),
                                          (int64_t)d.nblocks_mixed * sigbkg_threads(true));
  if (!(P.sorted && d.n >= 8 * t_max)) {
    const LeafDesc& L = P.leaf[ctx->sb.slot_v];
    sbtab_layout(theta_all[L.par[0]], theta_all[L.par[1]], theta_all[L.par[2]], L.lo, L.hi, H);
  }
  std::memcpy(theta_all + P.rec_off, &H, sizeof(H));
}

int theta_all_size(const gf_ctx* ctx) {
  const int np = (int)ctx->pars.size();
  if (ctx->compiled && ctx->use_sb)
    return std::max(np, ctx->prog.rec_off + (int)((sizeof(SBTabHdr) + 7) / 8));
  return np;
}

void fill_theta_all(const gf_ctx* ctx, const double* theta, double* out) {
  const int np = (int)ctx->pars.size();
  for (int i = 0; i < np; ++i) out[i] = ctx->pars[i].value;
  for (size_t k = 0; k < ctx->free_ids.size(); ++k) out[ctx->free_ids[k]] = theta[k];
}

int tick_prepare(gf_ctx* ctx) {
  DevState& d = ctx->dev;
  if (d.tick_desc) return d.tick_kind;
  if (!ctx->compiled || !d.theta || d.n <= 0) return 0;
  if (d.nconv > 0 || d.ngn > 0) return 0;  // tables / grid normalisations: per-fit evaluations
  if (ctx->is_tddp) return 0;
  CK(cudaSetDevice(ctx->device));
  if (!ctx->is_dalitz) {
    Fit1D F{};
    F.P = ctx->prog;
    for (int k = 0; k < d.nobs; ++k) F.cols.c[k] = d.cols[k];
    F.n = d.n;
    F.derived = d.derived;
    F.partials = d.partials;
    F.partials_norm = d.partials2;
    F.counter_ev = d.counters;
    F.counter_norm = d.counters + 1;
    F.analytic_only = ctx->has_grid ? 0 : 1;
    F.sbtab = ctx->use_sb ? d.sbtab : nullptr;
    // the signal + background form also gets its own event descriptor, after the Fit1D
    // (whose program the normalisation tick uses)
    const size_t off = round_up(sizeof(F), 256);
    CK(cudaMalloc(&d.tick_desc, off + sizeof(FitSB)));
    CK(cudaMemcpyAsync(d.tick_desc, &F, sizeof(F), cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->use_sb) {
      FitSB S{};
      S.D = ctx->sb;
      S.x = d.cols[ctx->prog.ins[ctx->prog.mix_leaf[0]].obs];
      S.n = d.n;
      S.derived = d.derived;
      S.partials = d.partials;
      S.counter = d.counters;
      S.sorted = ctx->prog.sorted;
      S.sbtab = d.sbtab;
      S.rec_off = ctx->prog.rec_off;
      CK(cudaMemcpyAsync(static_cast<char*>(d.tick_desc) + off, &S, sizeof(S),
                         cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    d.tick_kind = ctx->use_sb ? 3 : 1;
    return d.tick_kind;
  }
  // Dalitz: only with every shape fixed (Gram normalisation) and the caches built
  const DalitzPlan& D = ctx->dplan;
  for (int r = 0; r < D.nres; ++r)
    if (D.res[r].ev_cached < 0) return 0;
  if (!d.gram_valid) return 0;
  const bool mixed = ctx->precision == GF_MIXED;
  for (int r = 0; r < D.nres; ++r)
    if (!(d.ev_m0.size() == (size_t)D.nres && d.ev_m0[r] == d.h_theta[D.res[r].p_m0])) return 0;
  FitDz F{};
  F.D = D;
  F.s12 = d.cols[0];
  F.s13 = d.cols[1];
  F.sf = d.fcols;
  F.n = d.n;
  F.ev_cache = d.ev_cache;
  F.gram = d.gram;
  F.partials = d.partials;
  F.counter = d.counters;
  F.norm_scratch = d.norm_out;
  F.cache_wide = mixed ? 0 : 2;  // float2, or FP64 amplitudes as float pairs
  CK(cudaMalloc(&d.tick_desc, sizeof(F)));
  CK(cudaMemcpyAsync(d.tick_desc, &F, sizeof(F), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  d.tick_kind = 2;
  return 2;
}

int tick_finish(gf_ctx* ctx, const double* res, double* nll, double* grad) {
  const int nf = (int)ctx->free_ids.size();
  bool finite = std::isfinite(res[0]);
  for (int k = 0; k < nf; ++k) {
    grad[k] = res[1 + k];
    finite = finite && std::isfinite(grad[k]);
  }
  if (!finite) {
    *nll = INFINITY;
    return set_error(ctx, GF_ENONFINITE, "non-finite likelihood: some P_i <= 0 or not finite");
  }
  *nll = res[0];
  return GF_OK;
}

// A data set evaluated repeatedly (a fit) after gf_update_data gets sorted again.
static int resort_if_repeated(gf_ctx* ctx) {
  DevState& d = ctx->dev;
  if (!d.sorted && d.owns_cols && ++d.evals_since_load >= 2 && sort_eligible(ctx)) {
    CK(cudaSetDevice(ctx->device));
    return sort_events(ctx);
  }
  return GF_OK;
}

int evaluate(gf_ctx* ctx, const double* theta, double* nll, double* grad, bool fp64) {
  if (ctx->eval_in_flight)
    return set_error(ctx, GF_ESTATE, "an evaluation started by gf_nll_grad_start is not finished");
  int rc = resort_if_repeated(ctx);
  if (rc) return rc;
  rc = evaluate_async(ctx, theta, grad != nullptr, fp64);
  if (rc) return rc;
  return evaluate_finish(ctx, nll, grad, grad != nullptr);
}

}  // namespace gfi

extern "C" {

int gf_nll(gf_ctx* ctx, const double* theta, double* nll) {
  if (!ctx || !nll) return GF_EINVAL;
  int rc = ensure_compiled(ctx);
  if (rc) return rc;
  if (!theta && !ctx->free_ids.empty()) return GF_EINVAL;
  return evaluate(ctx, theta, nll, nullptr);
}

int gf_nll_grad(gf_ctx* ctx, const double* theta, double* nll, double* grad) {
  if (!ctx || !nll) return GF_EINVAL;
  int rc = ensure_compiled(ctx);
  if (rc) return rc;
  if (!ctx->free_ids.empty() && (!theta || !grad)) return GF_EINVAL;
  return evaluate(ctx, theta, nll, grad);
}

int gf_nll_grad_start(gf_ctx* ctx, const double* theta) {
  if (!ctx) return GF_EINVAL;
  if (ctx->eval_in_flight)
    return set_error(ctx, GF_ESTATE, "gf_nll_grad_start: an evaluation is already in flight");
  int rc = ensure_compiled(ctx);
  if (rc) return rc;
  if (!ctx->free_ids.empty() && !theta) return GF_EINVAL;
  rc = resort_if_repeated(ctx);
  if (rc) return rc;
  rc = evaluate_async(ctx, theta, true, false);
  if (rc) return rc;
  ctx->eval_in_flight = true;
  return GF_OK;
}

int gf_nll_grad_finish(gf_ctx* ctx, double* nll, double* grad) {
  if (!ctx || !nll) return GF_EINVAL;
  if (!ctx->eval_in_flight)
    return set_error(ctx, GF_ESTATE, "gf_nll_grad_finish: no evaluation in flight");
  if (!ctx->free_ids.empty() && !grad) return GF_EINVAL;
  ctx->eval_in_flight = false;
  return evaluate_finish(ctx, nll, grad, true);
}

static int logpdf_impl(gf_ctx* ctx, const double* theta, double* out, bool host) {
  if (!ctx || !out) return GF_EINVAL;
  int rc = ensure_compiled(ctx);
  if (rc) return rc;
  if (!theta && !ctx->free_ids.empty()) return GF_EINVAL;
  DevState& d = ctx->dev;
  CK(cudaSetDevice(ctx->device));
  rc = upload_theta(ctx, theta);
  if (rc) return rc;
  double* dst = out;
  if (host) CK(cudaMalloc(&dst, sizeof(double) * std::max<int64_t>(d.n, 1)));
  int launches = 0;
  if (ctx->is_tddp) {
    rc = tddp_enqueue(ctx, false, dst, &launches);
  } else if (ctx->is_dalitz) {
    int mode = 0;
    rc = dalitz_prepare(ctx, &mode, &launches, ctx->precision == GF_MIXED);
    if (rc == GF_OK) {
      DalitzBufs B = dalitz_bufs(ctx, dst);
      const bool mixed = ctx->precision == GF_MIXED;
      cudaError_t e = cudaSuccess;
      if (mode == DN_DIRECT) {
        const int ncell_blocks = (int)std::min<int64_t>(
            ((int64_t)ctx->dplan.nbx * ctx->dplan.nby + kThreads - 1) / kThreads,
            (int64_t)ctx->sm_count);  // a few cells per thread: amortise the block set-up
        e = launch_dalitz_norm_direct(ctx->dplan, false, false, d.theta, B, ncell_blocks,
                                      ctx->stream);
      }
      if (e == cudaSuccess)
        e = launch_dalitz_events(ctx->dplan, mixed, false, true, mode, d.theta, B, d.nblocks,
                                 ctx->stream);
      if (e != cudaSuccess) rc = cuda_fail(ctx, e, "launch_dalitz_events");
    }
  } else {
    const WeidCoef& W = weideman();
    if (ctx->has_grid) {
      const bool tab = ctx->use_sb && d.sbtab;
      cudaError_t e = launch_norm_1d(ctx->prog, d.prog, W, d.theta, d.partials2, d.counters + 1,
                                     d.derived, tab ? sbtab_hdr(ctx) : nullptr,
                                     tab ? d.sbtab : nullptr, sbtab_blocks(ctx), ctx->stream);
      if (e != cudaSuccess) rc = cuda_fail(ctx, e, "launch_norm_1d");
      if (rc == GF_OK) rc = enqueue_convs(ctx, nullptr);
    }
    Cols cols{};
    for (int k = 0; k < d.nobs; ++k) cols.c[k] = d.cols[k];
    if (rc == GF_OK && ctx->use_sb) {
      cudaError_t e = launch_sigbkg(ctx->sb, W, d.prog,
                                    d.cols[ctx->prog.ins[ctx->prog.mix_leaf[0]].obs], d.n,
                                    d.derived, d.partials, d.counters, d.result, dst,
                                    d.sorted ? d.perm : nullptr, false,
                                    ctx->precision == GF_MIXED,
                                    ctx->precision == GF_MIXED ? d.nblocks_mixed : d.nblocks,
                                    sbtab_hdr(ctx), d.sbtab, ctx->stream);
      if (e != cudaSuccess) rc = cuda_fail(ctx, e, "launch_sigbkg");
    } else if (rc == GF_OK) {
      cudaError_t e = launch_events_1d(ctx->prog, d.prog, W, cols, d.n, d.theta, d.derived, d.partials,
                                       d.counters, d.result, dst, d.sorted ? d.perm : nullptr,
                                       false, true,
                                       ctx->has_grid ? 0 : 1, d.nblocks, ctx->stream);
      if (e != cudaSuccess) rc = cuda_fail(ctx, e, "launch_events_1d");
    }
  }
  if (rc == GF_OK && host && d.n > 0) {
    cudaError_t e = cudaMemcpyAsync(out, dst, sizeof(double) * d.n, cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e != cudaSuccess) rc = cuda_fail(ctx, e, "copy log P");
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (host) cudaFree(dst);
  if (rc == GF_OK && e != cudaSuccess) rc = cuda_fail(ctx, e, "sync");
  return rc;
}

int gf_logpdf(gf_ctx* ctx, const double* theta, double* out) {
  return logpdf_impl(ctx, theta, out, true);
}
int gf_logpdf_device(gf_ctx* ctx, const double* theta, double* out_dev) {
  return logpdf_impl(ctx, theta, out_dev, false);
}

int gf_dalitz_gram(gf_ctx* ctx, const double* theta, double* G) {
  if (!ctx || !G) return GF_EINVAL;
  int rc = ensure_compiled(ctx);
  if (rc) return rc;
  if (!ctx->is_dalitz) return set_error(ctx, GF_EINVAL, "root is not a Dalitz node");
  if (!theta && !ctx->free_ids.empty()) return GF_EINVAL;
  DevState& d = ctx->dev;
  CK(cudaSetDevice(ctx->device));
  rc = upload_theta(ctx, theta);
  if (rc) return rc;
  const DalitzPlan& D = ctx->dplan;
  // columns of every resonance at this theta, then the Gram matrix
  int launches = 0;
  if (!d.mask_built) {
    CK(launch_dalitz_mask(D, d.inside, ctx->stream));
    d.mask_built = true;
  }
  std::vector<int> all(D.nres);
  for (int r = 0; r < D.nres; ++r) all[r] = r;
  CK(cudaMemcpyAsync(d.todo, all.data(), sizeof(int) * D.nres, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(launch_dalitz_grid_cols(D, d.theta, d.todo, D.nres, d.grid_cols, d.inside, ctx->stream));
  DalitzBufs B = dalitz_bufs(ctx, nullptr);
  CK(launch_dalitz_gram(D, B, ctx->stream));
  const int K = D.nres + 1;
  CK(cudaMemcpyAsync(G, d.gram, sizeof(double) * 2 * K * K, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int r = 0; r < D.nres; ++r) {
    d.col_m0[r] = d.h_theta[D.res[r].p_m0];
    d.col_g0[r] = d.h_theta[D.res[r].p_g0];
  }
  d.gram_valid = true;
  (void)launches;
  return GF_OK;
}

int gf_last_eval_times(gf_ctx* ctx, double* total_ms, double* stream_ms) {
  if (!ctx) return GF_EINVAL;
  if (total_ms) *total_ms = ctx->last_ms;
  if (stream_ms) *stream_ms = ctx->last_stream_ms;
  return GF_OK;
}

// The range-check flag of spare set q (slots 61, 62 of the mapped result block).
static volatile int* stage_flag_host(DevState& d, int q) {
  return reinterpret_cast<volatile int*>(d.h_result + 61 + q);
}

// Wait for the oldest prefetch still in flight and forget it (its buffers stay allocated).
static int drop_oldest(gf_ctx* ctx) {
  DevState& d = ctx->dev;
  if (d.npend == 0) return GF_OK;
  const int q = d.pend[0];
  d.stage_src[q].clear();
  for (int k = 1; k < d.npend; ++k) d.pend[k - 1] = d.pend[k];
  d.npend--;
  CK(cudaEventSynchronize(d.ev_staged[q]));
  return GF_OK;
}

// ... and every one of them.
static int drop_staged(gf_ctx* ctx) {
  while (ctx->dev.npend > 0) {
    const int rc = drop_oldest(ctx);
    if (rc) return rc;
  }
  return GF_OK;
}

// The oldest prefetched set becomes the context's data: its copy and range check ran on
// the copy stream during earlier work, so this is a swap of two buffer sets.  The new
// events are in the caller's order (the strided event loop; a set evaluated repeatedly is
// sorted again from its second evaluation, as after gf_update_data).
static int swap_staged(gf_ctx* ctx) {
  DevState& d = ctx->dev;
  const int q = d.pend[0];
  d.stage_src[q].clear();
  for (int k = 1; k < d.npend; ++k) d.pend[k - 1] = d.pend[k];
  d.npend--;
  CK(cudaEventSynchronize(d.ev_staged[q]));
  volatile int* sflag = stage_flag_host(d, q);
  if (*sflag) {
    *sflag = 0;
    return set_error(ctx, GF_EINVAL, "gf_update_data: an event of the prefetched set lies outside "
                                     "its range (the set was not loaded)");
  }
  std::swap(d.cols, d.stage[q]);
  std::swap(d.cur_set, d.stage_id[q]);
  const int rc = mark_unsorted(ctx);  // the kernels read the flag from the device program
  if (rc) return rc;
  if (d.tick_desc) {  // the serving descriptor holds the old column pointers
    cudaStreamSynchronize(ctx->stream);
    cudaFree(d.tick_desc);
    d.tick_desc = nullptr;
    d.tick_kind = 0;
  }
  return GF_OK;
}

int gf_prefetch_data(gf_ctx* ctx, int64_t n, const double* const* cols) {
  if (!ctx || !cols) return GF_EINVAL;
  DevState& d = ctx->dev;
  if (!d.owns_cols || !d.theta) return set_error(ctx, GF_ESTATE, "no data set owned by the context");
  if (n != d.n) return set_error(ctx, GF_EINVAL, "gf_prefetch_data: n must equal the loaded size");
  if (d.binned || ctx->is_dalitz || ctx->is_tddp)
    return set_error(ctx, GF_EINVAL, "gf_prefetch_data: 1D unbinned data sets only");
  for (int k = 0; k < d.nobs; ++k)
    if (!cols[k]) return GF_EINVAL;
  int rc = ensure_compiled(ctx);
  if (rc) return rc;
  CK(cudaSetDevice(ctx->device));
  if (d.npend == DevState::kStage) {  // the queue is full: the oldest is never loaded
    rc = drop_oldest(ctx);
    if (rc) return rc;
  }
  if (!d.copy_stream) {
    CK(cudaStreamCreateWithFlags(&d.copy_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&d.check_stream, cudaStreamNonBlocking));
    for (int q = 0; q < DevState::kStage; ++q) {
      CK(cudaEventCreateWithFlags(&d.ev_copied[q], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&d.ev_staged[q], cudaEventDisableTiming));
    }
    CK(cudaEventCreateWithFlags(&d.ev_free, cudaEventDisableTiming));
  }
  int q = 0;  // a spare set holding no prefetch
  while (!d.stage_src[q].empty()) ++q;
  const size_t bytes = round_up((size_t)std::max<int64_t>(n + 2, 2) * 8, 256);
  while ((int)d.stage[q].size() < d.nobs) {
    double* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return set_error(ctx, GF_ENOMEM, "gf_prefetch_data: device allocation of the staging buffers failed");
    }
    d.stage[q].push_back(p);
    CK(cudaMemsetAsync(p, 0, bytes, d.copy_stream));
  }
  // the spare buffers may still be read by work queued on the compute stream
  CK(cudaEventRecord(d.ev_free, ctx->stream));
  CK(cudaStreamWaitEvent(d.copy_stream, d.ev_free, 0));
  *stage_flag_host(d, q) = 0;
  for (int k = 0; k < d.nobs; ++k)
    if (n > 0)
      CK(cudaMemcpyAsync(d.stage[q][k], cols[k], sizeof(double) * n, cudaMemcpyHostToDevice,
                         d.copy_stream));
  Cols c{};
  double lo[kMaxObs], hi[kMaxObs];
  for (int k = 0; k < d.nobs; ++k) {
    c.c[k] = d.stage[q][k];
    lo[k] = ctx->obs[d.obs_ids[k]].lo;
    hi[k] = ctx->obs[d.obs_ids[k]].hi;
  }
  // the check on its own stream behind the copy: the copy stream goes on to the next
  // set's copy while the check waits for SMs the evaluation holds
  CK(cudaEventRecord(d.ev_copied[q], d.copy_stream));
  CK(cudaStreamWaitEvent(d.check_stream, d.ev_copied[q], 0));
  CK(launch_check_range(c, d.nobs, n, lo, hi, reinterpret_cast<int*>(d.result + 61 + q),
                        d.check_stream));
  CK(cudaEventRecord(d.ev_staged[q], d.check_stream));
  d.stage_src[q].assign(cols, cols + d.nobs);
  d.pend[d.npend++] = q;
  return GF_OK;
}

int gf_update_data(gf_ctx* ctx, int64_t n, const double* const* cols) {
  if (!ctx || !cols) return GF_EINVAL;
  DevState& d = ctx->dev;
  if (!d.owns_cols || !d.theta) return set_error(ctx, GF_ESTATE, "no data set owned by the context");
  if (n != d.n) return set_error(ctx, GF_EINVAL, "gf_update_data: n must equal the loaded size");
  if (d.binned) return set_error(ctx, GF_EINVAL, "gf_update_data: binned data go through gf_set_data");
  if (d.npend > 0) {
    // the columns of a pending prefetch: the ones staged before it are never loaded
    int at = -1;
    for (int j = 0; j < d.npend && at < 0; ++j) {
      bool same = true;
      for (int k = 0; k < d.nobs; ++k) same = same && d.stage_src[d.pend[j]][k] == cols[k];
      if (same) at = j;
    }
    CK(cudaSetDevice(ctx->device));
    for (int j = 0; j < at; ++j) {
      const int rd = drop_oldest(ctx);
      if (rd) return rd;
    }
    if (at >= 0) return swap_staged(ctx);
    const int rd = drop_staged(ctx);  // another set: the prefetched ones are not used
    if (rd) return rd;
  }
  d.tddp_ready = false;  // per-event amplitudes of the new events
  int rc = ensure_compiled(ctx);
  if (rc) return rc;
  CK(cudaSetDevice(ctx->device));
  rc = mark_unsorted(ctx);  // the new events arrive in the caller's order
  if (rc) return rc;
  for (int k = 0; k < d.nobs; ++k)
    if (!cols[k]) return GF_EINVAL;
  if (ctx->is_tddp) {
    // the checks gf_set_data makes, on the host copies, before any event is replaced
    for (int64_t i = 0; i < n; ++i) {
      if (!(cols[3][i] > 0.0))
        return set_error(ctx, GF_EINVAL, "event " + std::to_string(i) + ": sigma_t must be > 0");
      if (!dalitz_inside_host(ctx->tplan.D, cols[0][i], cols[1][i]))
        return set_error(ctx, GF_EINVAL,
                         "event " + std::to_string(i) + " outside the Dalitz kinematic region");
    }
  }
  for (int k = 0; k < d.nobs; ++k) {
    if (n > 0)
      CK(cudaMemcpyAsync(d.cols[k], cols[k], sizeof(double) * n, cudaMemcpyHostToDevice,
                         ctx->stream));
  }
  if (ctx->is_dalitz) {
    CK(launch_dalitz_check(ctx->dplan, d.cols[0], d.cols[1], n, d.flag, ctx->stream));
    if (d.fcols)
      CK(launch_dalitz_fcols(ctx->dplan, d.cols[0], d.cols[1], n, d.fcols, ctx->stream));
    for (auto& v : d.ev_m0) v = NAN;  // per-event caches hold the old events
    for (auto& v : d.ev64_m0) v = NAN;
  } else {
    Cols c{};
    double lo[kMaxObs], hi[kMaxObs];
    for (int k = 0; k < d.nobs; ++k) {
      c.c[k] = d.cols[k];
      lo[k] = ctx->obs[d.obs_ids[k]].lo;
      hi[k] = ctx->obs[d.obs_ids[k]].hi;
    }
    CK(launch_check_range(c, d.nobs, n, lo, hi, d.flag, ctx->stream));
  }
  return GF_OK;
}

int gf_set_metric(gf_ctx* ctx, int metric) {
  if (!ctx) return GF_EINVAL;
  if (metric != GF_METRIC_NLL && metric != GF_METRIC_BINNED_NLL && metric != GF_METRIC_CHISQ)
    return set_error(ctx, GF_EINVAL, "unknown metric");
  if (ctx->metric != metric) {
    ctx->metric = metric;
    ctx->compiled = false;  // recompiled (and graphs re-captured) at the next call
  }
  return GF_OK;
}

int gf_set_mixture_path(gf_ctx* ctx, int enable) {
  if (!ctx) return GF_EINVAL;
  if (ctx->mixture_path != (enable != 0)) {
    ctx->mixture_path = enable != 0;
    ctx->compiled = false;  // recompiled (and graphs re-captured) at the next call
  }
  return GF_OK;
}

int gf_set_event_sort(gf_ctx* ctx, int enable) {
  if (!ctx) return GF_EINVAL;
  ctx->event_sort = enable != 0;
  return GF_OK;
}

int gf_set_graphs(gf_ctx* ctx, int enable) {
  if (!ctx) return GF_EINVAL;
  ctx->graphs = enable != 0;
  return GF_OK;
}

int gf_last_eval_graph(gf_ctx* ctx, int* replayed, char* why_not, size_t n) {
  if (!ctx) return GF_EINVAL;
  if (replayed) *replayed = ctx->last_graph ? 1 : 0;
  if (why_not && n > 0) std::snprintf(why_not, n, "%s", ctx->dev.graph_why.c_str());
  return GF_OK;
}

int gf_last_eval_stats(gf_ctx* ctx, double* kernel_ms, int* launches) {
  if (!ctx) return GF_EINVAL;
  if (kernel_ms) *kernel_ms = ctx->last_ms;
  if (launches) *launches = ctx->last_launches;
  return GF_OK;
}

}  // extern "C"
