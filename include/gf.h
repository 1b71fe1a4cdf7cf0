/*
 * gf.h -- C ABI of the GB300 (sm_103a) unbinned maximum-likelihood engine.
 *
 * The calls follow the paper's statement of a fit (Andreassen et al., "GooFit: A
 * library for massively parallelising maximum-likelihood fits", arXiv:1311.1753,
 * Sec. 2): declare observables and fit parameters (Variable), build the PDF
 * (GooPdf and its combinations, Sec. 3), load an unbinned dataset
 * (UnbinnedDataSet / setData), evaluate the likelihood and fit (FitManager).
 *
 * Conventions for every call:
 *  - Return value: GF_OK (0) or a negative GF_E* code; nothing aborts, and no GPU
 *    error is raised on purpose.  gf_last_error() gives a message for the last failure
 *    on a context.
 *  - Pointers are plain host pointers unless the name says "_device"; arrays passed
 *    in are copied, so the caller keeps ownership and may free them after the call.
 *  - A context (gf_ctx) owns every object created through it (observables,
 *    parameters, PDF nodes, device memory, CUDA stream).  A context is not
 *    thread-safe: use one per host thread.
 *  - Identifiers (observable, parameter, node) are small non-negative ints scoped
 *    to their context.
 */
#ifndef GF_H
#define GF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------- */
#define GF_OK 0
#define GF_EINVAL (-1)      /* bad argument, unknown id, cycle, event out of range   */
#define GF_ENOMEM (-2)      /* host or device allocation failed                      */
#define GF_ECUDA (-3)       /* a CUDA runtime call failed                            */
#define GF_ENONFINITE (-4)  /* some P_i <= 0 or non-finite: nll set to +inf          */
#define GF_ENOCONV (-5)     /* minimiser stopped without meeting the EDM tolerance   */
#define GF_ETIMEOUT (-6)    /* a bounded wait ran out (server)                       */
#define GF_ESTATE (-7)      /* call out of order (e.g. evaluate before gf_set_data)  */

/* ---- precision modes -------------------------------------------------------------- */
/* GF_FP64: FP64-accurate results.  On GB300 the per-event and per-cell arithmetic runs
 *   as double-float (pairs of FP32 values, 48-bit significands, on the FP32 pipe), with
 *   exact FP64 differences of data and constants and an FP64 re-evaluation of events
 *   outside the float exponent range; per event it meets 1e-12 relative to the FP64
 *   definition, the NLL 1e-9 relative (the library's tests).
 * GF_MIXED: per-event PDF and amplitude arithmetic in FP32; the log-sum across threads
 *   and blocks, the normalisation integrals and (1D trees) the Faddeeva function of the
 *   Voigtian stay FP64-accurate.  Results carry FP32 rounding (stated by the tests). */
#define GF_FP64 0
#define GF_MIXED 1

typedef struct gf_ctx gf_ctx;
typedef struct gf_dataset gf_dataset;

/* ---- context -------------------------------------------------------------------- */
/* Create a context on CUDA device `device` with precision GF_FP64 or GF_MIXED.
 * The context creates its own CUDA stream.  *out is NULL on failure. */
int gf_create(gf_ctx** out, int device, int precision);
/* Release every object, device buffer and stream of the context.  NULL is a no-op. */
int gf_destroy(gf_ctx* ctx);
/* Run all of the context's GPU work on `stream` (a cudaStream_t on the context's
 * device, owned by the caller and alive until gf_destroy or another gf_set_stream);
 * NULL returns to the context's own stream. */
int gf_set_stream(gf_ctx* ctx, void* stream);
/* Text for a status code (static storage). */
const char* gf_strerror(int code);
/* Copy the message of the context's last failure into buf (NUL-terminated). */
int gf_last_error(gf_ctx* ctx, char* buf, size_t n);

/* ---- variables (Sec. 2: the two uses of Variable) -------------------------------- */
/* Observable with range [lo, hi] (Listing 1: Variable(name, lo, hi)); lo < hi. */
int gf_observable(gf_ctx* ctx, const char* name, double lo, double hi, int* id);
/* Fit parameter (Listing 1: Variable(name, init, step, lo, hi)).  lo < hi bounds the
 * parameter with MINUIT's sine transform; lo == hi == 0 leaves it unbounded.  step is
 * the minimiser's initial scale (> 0). */
int gf_parameter(gf_ctx* ctx, const char* name, double init, double step, double lo, double hi,
                 int* id);
/* Fix (1) or release (0) a parameter.  Fixed parameters keep their value and are not
 * part of theta. */
int gf_set_fixed(gf_ctx* ctx, int par, int fixed);
/* Set a parameter's current value (the start value of the next gf_fit). */
int gf_set_value(gf_ctx* ctx, int par, double value);
int gf_get_value(gf_ctx* ctx, int par, double* value);
/* Number of free parameters and their ids in theta order (declaration order).
 * ids may be NULL; otherwise it has room for *n entries. */
int gf_free_params(gf_ctx* ctx, int* n, int* ids);

/* ---- PDF nodes (Sec. 3, Listing 3-4) ---------------------------------------------
 * Leaves are normalised on their observable's range: analytically where a closed form
 * exists (exponential, Gaussian, polynomial), otherwise by the midpoint rule on the
 * node's grid (default 10,000 bins; gf_set_norm_grid).  Arguments named after
 * parameters are parameter ids. */
/* e^{alpha x} (Listing 1, ExpPdf). */
int gf_pdf_exp(gf_ctx* ctx, int obs, int alpha, int* node);
/* exp(-(x-mu)^2/(2 sigma^2)) (Listing 3, GaussianPdf). */
int gf_pdf_gauss(gf_ctx* ctx, int obs, int mu, int sigma, int* node);
/* Voigtian: Breit-Wigner of FWHM `width` convolved with a Gaussian of std `sigma`
 * (Sec. 4: the line shape of the D*+ width fit), Re w(z)/(sigma sqrt(2 pi)),
 * z = (x - mu + i width/2)/(sigma sqrt 2). */
int gf_pdf_voigt(gf_ctx* ctx, int obs, int mu, int sigma, int width, int* node);
/* Threshold shape (x - x0)^power exp(-c (x - x0)) for x > x0, 0 below. */
int gf_pdf_threshold(gf_ctx* ctx, int obs, int x0, int power, int c, int* node);
/* Polynomial sum_k coef[k] x^k, ncoef <= 8. */
int gf_pdf_poly(gf_ctx* ctx, int obs, int ncoef, const int* coefs, int* node);
/* Relativistic Breit-Wigner line shape (Sec. 4: the P-wave D*+ line fitted in the D*+ - D0
 * mass difference) in x = m - shift:
 *   f = m Gamma(m) / ((m0^2 - m^2)^2 + m0^2 Gamma(m)^2),  m = x + shift, m0 = dm0 + shift,
 *   Gamma(m) = gamma0 (q/q0)^{2 spin + 1} (m0/m) B(z0)/B(z),
 * q the break-up momentum of masses ma, mb at m, z = (q radius)^2, Blatt-Weisskopf
 * B = 1, 1 + z, 9 + 3z + z^2 for spin 0, 1, 2; zero at or below ma + mb.  Normalised on
 * the node's grid.  shift, ma, mb and radius must be fixed parameters (GF_EINVAL at the
 * first evaluation otherwise). */
int gf_pdf_relbw(gf_ctx* ctx, int obs, int dm0, int gamma0, int shift, int ma, int mb,
                 int radius, int spin, int* node);
/* ConvolutionPdf (Sec. 3): the model node (over obs) convolved with the resolution node,
 * whose leaves use one residual observable r (declared like any observable; its range
 * [rlo, rhi] is the resolution's support and is not a data column).  Numerically, on a
 * lattice of L bins of obs's range (gf_set_norm_grid(node, L), default 1000, at most
 * 65536; h = (hi - lo)/L): C_i = h sum_k R(k h) M(x_i - k h) over the offsets k h in
 * [rlo, rhi] (at most 8193), C linear between lattice points, P = C / N with N the
 * trapezoid integral h (C_0/2 + C_1 + ... + C_L/2).  Model and resolution are normalised
 * on their own ranges (the model is evaluated outside its range where the lattice needs
 * it).  At most 2 convolutions per tree, none nested, at most 8 free parameters in the
 * model and resolution together. */
int gf_pdf_conv(gf_ctx* ctx, int obs, int model, int resolution, int* node);
/* MappedPdf (Sec. 3): nodes[k] on [b_{k-1}, b_k) of obs's range (b_{-1} = lo; the last
 * interval is closed at hi), bounds the n - 1 interior boundaries as parameter ids (fixed;
 * increasing), 2 <= n <= 4.  Each component is normalised on its own range as usual; the
 * piecewise result is normalised by the midpoint rule on the node's grid
 * (gf_set_norm_grid, default 10,000 bins). */
int gf_pdf_mapped(gf_ctx* ctx, int obs, int n, const int* nodes, const int* bounds, int* node);
/* CompositePdf (Sec. 3): f(g(x)) with g the core leaf (over obs) and f the shell leaf (an
 * exponential, Gaussian or polynomial node over any observable, whose range is ignored),
 * both as unnormalised shapes; the result is normalised by the midpoint rule on the node's
 * grid (default 10,000 bins).  A tree holds at most 2 MappedPdf/CompositePdf nodes, not
 * nested in one another or in a convolution, with at most 8 free parameters each. */
int gf_pdf_composite(gf_ctx* ctx, int obs, int core, int shell, int* node);
/* AddPdf (Sec. 3): sum_{k<n-1} f_k P_k + (1 - sum f) P_{n-1}; fracs has n-1 ids, n <= 8. */
int gf_pdf_add(gf_ctx* ctx, int n, const int* nodes, const int* fracs, int* node);
/* ProdPdf (Sec. 3, Listing 2): prod_k P_k; the factors must use distinct observables. */
int gf_pdf_prod(gf_ctx* ctx, int n, const int* nodes, int* node);

/* Three-body decay M -> 1 2 3 on the Dalitz plot (Sec. 4).  Observables are
 * s12 = m12^2 and s13 = m13^2 (their declared ranges are ignored: the kinematic
 * region decides).  Amplitude A = a_NR + sum_r c_r F_L S_L BW_r with a fixed
 * non-resonant a_NR = 1, c_r = re + i im, relativistic Breit-Wigner
 * BW = 1/(m0^2 - s - i m0 Gamma(m)), Gamma(m) = Gamma0 (q/q0)^{2L+1} (m0/m) F_L^2,
 * Blatt-Weisskopf F_L at the resonance vertex with radius R, Zemach spin factors S_L;
 * P = |A|^2, normalised on a grid of cell centres inside the region (512 x 512 by
 * default). */
typedef struct {
  double M, m1, m2, m3; /* parent and daughter masses (GeV) */
  double R;             /* Blatt-Weisskopf radius (GeV^-1) */
} gf_dalitz_kin;
typedef struct {
  int channel;          /* 0: (12) bachelor 3; 1: (13) bachelor 2; 2: (23) bachelor 1 */
  int spin;             /* 0, 1 or 2 */
  int mass, width;      /* parameter ids of m0, Gamma0 */
  int re, im;           /* parameter ids of the coefficient */
} gf_resonance;
int gf_pdf_dalitz(gf_ctx* ctx, int obs12, int obs13, const gf_dalitz_kin* kin, int nres,
                  const gf_resonance* res, int* node);
/* Time-dependent Dalitz model (Sec. 4: the D0 -> pi+ pi- pi0 mixing fit): the amplitude
 * model of gf_pdf_dalitz (particles 1 and 2 CP conjugates, m1 = m2) for D0 (A at
 * (s12, s13)) and D0bar (B, the same sum at (s12, s23)), with the decay
 * time t and its per-event uncertainty sigma_t:
 *   I = 1/2 (|A|^2 + |B|^2) Tch + 1/2 (|A|^2 - |B|^2) Tc + Re(A* B) Tsh - Im(A* B) Ts,
 * the time factors e^{-t/tau} {cosh(y t/tau), cos(x t/tau), sinh(y t/tau),
 * sin(x t/tau)} (t >= 0) each convolved with a Gaussian of width scale * sigma_t.
 * Normalised over the Dalitz grid (gf_set_norm_grid; default 256 x 256 cells) and all t;
 * conditional on sigma_t unless gf_tddp_sigt_density adds its density.  tau, x, y, scale
 * are parameter ids.  Resonance masses and widths may be free: the per-event amplitudes and
 * their derivatives are then recomputed when a shape changes and N by a direct pass over
 * the cells at each evaluation (fixed shapes: once per data load, N from grid sums).
 * The data set holds the columns s12, s13, t, sigma_t in this order (sigma_t > 0; every
 * event inside the
 * kinematic region, else GF_EINVAL from gf_set_data / gf_update_data).  FP64-accurate in
 * both precision modes: the time dependence in FP64, the amplitude algebra in
 * double-float pairs. */
int gf_pdf_tddp(gf_ctx* ctx, int obs12, int obs13, int obs_t, int obs_sigt,
                const gf_dalitz_kin* kin, int nres, const gf_resonance* res, int tau, int x,
                int y, int scale, int* node);
/* The decay-time uncertainty's density of a time-dependent Dalitz node (Sec. 4: the
 * mixing fit's sigma_t distribution varies across the Dalitz plot): the PDF becomes
 * I/N x D(sigma_t | s12, s13) with
 *   D = lam^2 sigma_t e^{-lam sigma_t} / Z,  Z = g(lam lo) - g(lam hi),  g(a) = e^{-a}(1 + a),
 *   lam = exp(b0 + b1 (s12 - sc) + b2 (s13 - sc)),  sc = (M^2 + m1^2 + m2^2 + m3^2)/3,
 * a Gamma distribution of shape 2 truncated to the sigma_t observable's range [lo, hi]
 * (lo > 0) whose rate varies over the plot; b0, b1, b2 are parameter ids.  D integrates
 * to one over sigma_t at every point, so the product is normalised.  Without this call the
 * likelihood is conditional on sigma_t. */
int gf_tddp_sigt_density(gf_ctx* ctx, int node, int b0, int b1, int b2);
/* Grid of the node's numerical normalisation: nbins_x bins for a 1D leaf, the lattice
 * of a convolution, or nbins_x x nbins_y cells for a Dalitz node. */
int gf_set_norm_grid(gf_ctx* ctx, int node, int nbins_x, int nbins_y);
/* 1 if (s12, s13) lies inside the kinematic region of the Dalitz node, else 0, for n
 * points (host arrays). */
int gf_dalitz_inside(gf_ctx* ctx, int node, int64_t n, const double* s12, const double* s13,
                     int8_t* out);

/* ---- data (Sec. 2: UnbinnedDataSet, addEvent, setData) ------------------------------ */
/* Host-side dataset over nobs observables (ids copied). */
int gf_dataset_create(gf_ctx* ctx, int nobs, const int* obs, gf_dataset** ds);
/* Append n events given as one host column per observable (cols[k][i] is observable
 * obs[k] of event i).  Any event outside an observable's range (or, for a Dalitz
 * model's observables, outside the kinematic region at gf_set_data) makes the call
 * fail with GF_EINVAL and adds nothing. */
int gf_dataset_add_events(gf_dataset* ds, int64_t n, const double* const* cols);
int64_t gf_dataset_size(const gf_dataset* ds);
int gf_dataset_destroy(gf_dataset* ds);
/* Binned data set (Sec. 4: the D*+ line-width fit is a binned fit; Sec. 2: the fit's
 * metric is separate from the PDF's evaluation).  Each observable obs[k]'s range is
 * divided into nbins[k] equal bins; counts[b] >= 0 is the content of bin b, row-major
 * over the observables (the last one fastest), prod(nbins) entries; errors is NULL or
 * the uncertainty sigma_b > 0 of each bin (used by GF_METRIC_CHISQ; NULL: sigma_b^2 =
 * max(counts[b], 1)).  The bin centres become the data set's events; bin b's expected
 * content is nu_b = N V P(x_b) with N = sum_b counts[b] and V the bin volume.  Arrays are
 * copied.  Errors: GF_EINVAL for a bad id, nbins < 1, more than 2^31 bins, a negative or
 * non-finite count, or a non-positive error; gf_dataset_add_events on it fails. */
int gf_dataset_create_binned(gf_ctx* ctx, int nobs, const int* obs, const int* nbins,
                             const double* counts, const double* errors, gf_dataset** ds);

/* The fit's metric (Sec. 2: FitManager's metric, summed over events or bins):
 *  GF_METRIC_NLL         -sum_i w_i log P(x_i); w_i = 1 for unbinned data, the bin
 *                        content for binned data (multinomial likelihood).  Default.
 *  GF_METRIC_BINNED_NLL  sum_b (nu_b - n_b log nu_b): Poisson likelihood of the bin
 *                        contents (the constant sum log n_b! is left out).  Binned only.
 *  GF_METRIC_CHISQ       sum_b (n_b - nu_b)^2 / sigma_b^2.  Binned only.
 * gf_nll, gf_nll_grad and gf_fit then return / minimise this quantity; the error
 * definition of gf_fit defaults to 1 for GF_METRIC_CHISQ and 0.5 otherwise.  Takes effect
 * at the next evaluation; a binned metric without binned data gives GF_EINVAL there. */
#define GF_METRIC_NLL 0
#define GF_METRIC_BINNED_NLL 1
#define GF_METRIC_CHISQ 2
int gf_set_metric(gf_ctx* ctx, int metric);

/* Compile the tree rooted at `root`, copy the dataset's columns to device memory
 * (structure of arrays, 256-byte aligned, padded), and invalidate the normalisation
 * caches.  The dataset stays owned by the caller. */
int gf_set_data(gf_ctx* ctx, int root, const gf_dataset* ds);
/* As gf_set_data, but the n events are already in device memory: dev_cols[k] is a
 * device pointer to n doubles (observable obs[k]), 16-byte aligned, owned by the caller
 * and alive while the context uses it.  Nothing is copied and no range check is made. */
int gf_set_data_device(gf_ctx* ctx, int root, int nobs, const int* obs, int64_t n,
                       const double* const* dev_cols);

/* Replace the events of the loaded data set (same n, same observables) by new host
 * columns (cols[k] has n doubles; pinned memory makes the copy asynchronous).  The copy
 * is queued on the context's stream; the events are checked on the device against the
 * observable ranges (Dalitz: the kinematic region) and the next evaluation returns
 * GF_EINVAL if any is outside.  The per-event caches are rebuilt at that evaluation. */
int gf_update_data(gf_ctx* ctx, int64_t n, const double* const* cols);
/* (Binned data sets are replaced with gf_set_data; gf_update_data rejects them.  For the
 * time-dependent Dalitz model the kinematic region and sigma_t > 0 are checked on the
 * host, as gf_set_data does, and GF_EINVAL is returned with no event replaced.) */
/* Start loading the NEXT events of a 1D unbinned data set owned by the context (same n and
 * observables; cols[k] n doubles in host memory, pinned for an asynchronous copy) while
 * the current events are still being evaluated: the columns are copied on an internal
 * copy stream into a second device buffer set and checked against the observable ranges
 * there.  Returns at once.  A later gf_update_data with the same column pointers (cols[k]
 * identical) makes them the context's events by swapping the two buffer sets: no copy at
 * that call.  The new events are in the caller's order, as after gf_update_data (a data
 * set evaluated repeatedly is sorted again from its second evaluation).  The host columns
 * must stay unchanged until that gf_update_data returns.  A range error is reported by
 * that gf_update_data (GF_EINVAL; the prefetched set is not loaded, the loaded one stays).
 * Up to two prefetches may wait, copied one after the other: gf_update_data with the
 * columns of one of them loads it and drops the ones staged before it; a third
 * gf_prefetch_data drops the oldest; gf_update_data with other pointers or gf_set_data
 * waits for them and drops them all.  The evaluation graphs of the three buffer sets are
 * kept, so rotating sets does not re-capture them.  Device memory: up to two more copies
 * of the columns.
 * Dalitz, time-dependent Dalitz and binned data sets: GF_EINVAL; no data set owned:
 * GF_ESTATE. */
int gf_prefetch_data(gf_ctx* ctx, int64_t n, const double* const* cols);

/* ---- evaluation (Sec. 2: evaluate and metric, summed over events) ------------------ */
/* NLL(theta) = -sum_i log P(x_i; theta) with P normalised (or the context's binned
 * metric, gf_set_metric), at theta = the free parameters in gf_free_params order
 * (external units).  Blocking: returns when the value is on the host.  Non-finite
 * result: *nll = +inf, GF_ENONFINITE. */
int gf_nll(gf_ctx* ctx, const double* theta, double* nll);
/* NLL and its gradient over theta from the same event pass. */
int gf_nll_grad(gf_ctx* ctx, const double* theta, double* nll, double* grad);
/* The same evaluation in two halves, so that the host can work while the GPU computes
 * (Sec. 2's evaluation, pipelined with data loading).  gf_nll_grad_start queues the
 * evaluation at theta on the context's stream and returns; gf_nll_grad_finish waits for
 * it and returns what gf_nll_grad would have returned (the same bits).  Between the two
 * the caller may load the next events with gf_update_data (a swap with a prefetched set,
 * or a copy queued behind the evaluation) and queue more with gf_prefetch_data (its copy
 * waits for the queued evaluation before overwriting a buffer set it reads): the queued
 * evaluation keeps the events it started with.  One evaluation per context at a time:
 * until gf_nll_grad_finish, a second start and every call that evaluates or sets new
 * parameters or a new data set (gf_nll, gf_nll_grad, gf_logpdf, gf_fit, gf_set_data,
 * ...) returns GF_ESTATE; gf_nll_grad_finish without a start returns GF_ESTATE. */
int gf_nll_grad_start(gf_ctx* ctx, const double* theta);
int gf_nll_grad_finish(gf_ctx* ctx, double* nll, double* grad);
/* Per-event log P_i at theta into out (host array of n doubles, event order). */
int gf_logpdf(gf_ctx* ctx, const double* theta, double* out);
/* Same into a device array of n doubles. */
int gf_logpdf_device(gf_ctx* ctx, const double* theta, double* out_dev);
/* The Dalitz node's normalisation Gram matrix G (row-major (nres+1)^2 complex as
 * interleaved re, im; index 0 is a_NR) at theta: N = c^H G c.  Fit fractions follow
 * as |c_r|^2 G_rr / N. */
int gf_dalitz_gram(gf_ctx* ctx, const double* theta, double* G);

/* ---- fit (Sec. 2: FitManager + Migrad, here a quasi-Newton of this library) -------- */
typedef struct {
  double tol;      /* EDM tolerance (default 1e-6 when <= 0) */
  int max_calls;   /* evaluation budget (default 5000 when <= 0) */
  int use_grad;    /* 1: fused analytic gradient; 0: central differences of gf_nll */
  double up;       /* error definition; <= 0: 1 for GF_METRIC_CHISQ, else 0.5 */
  int hesse;       /* 1: covariance from the Hessian by differences of the gradient */
  int refine;      /* GF_MIXED contexts: 1 (default when opts is NULL) runs BFGS on the FP32
                      likelihood to EDM < max(tol, 1) (or until its rounding noise stops
                      the line search), then continues in FP64 from that point and
                      inverse-Hessian estimate to EDM < tol; errors from the FP32
                      Hessian.  0: FP32 only. */
} gf_fit_opts;
typedef struct {
  double nll;      /* NLL at the minimum */
  double edm;      /* estimated distance to minimum */
  int n_calls;     /* likelihood evaluations */
  int n_iter;      /* quasi-Newton iterations */
  int status;      /* GF_OK or GF_ENOCONV */
  double* theta;   /* caller-allocated, n_free: fitted values (external units) */
  double* err;     /* caller-allocated, n_free, or NULL: parabolic errors */
  double* cov;     /* caller-allocated, n_free^2, or NULL: covariance matrix */
  int n_calls_fast; /* of n_calls, those made on the FP32 likelihood (refined fits) */
} gf_fit_result;
/* Minimise from the parameters' current values; the fitted values become the current
 * values.  Returns the same status as res->status. */
int gf_fit(gf_ctx* ctx, const gf_fit_opts* opts, gf_fit_result* res);

/* ---- fit server (continuous batching of many fits) ----------------------------------- */
typedef struct gf_server gf_server;
typedef struct {
  int device;
  int precision;        /* GF_FP64 or GF_MIXED for every admitted fit */
  size_t mem_budget;    /* bytes of device memory the resident fits may hold */
  int max_slots;        /* maximum number of fits resident at once */
  double wait_timeout_s;/* bound on any internal wait (default 60 s) */
} gf_server_opts;
/* Start a server with its worker thread. */
int gf_server_create(const gf_server_opts* opts, gf_server** out);
/* Submit a fit: `model` is a context holding observables, parameters and the PDF
 * tree (no data needed); `ds` the events; `root` the PDF node.  The server takes
 * ownership of both (it destroys them when the fit is done); the request is admitted
 * when a slot and enough of the memory budget are free.  ticket identifies it. */
int gf_server_submit(gf_server* srv, gf_ctx* model, gf_dataset* ds, int root,
                     const gf_fit_opts* opts, uint64_t* ticket);
/* Non-blocking poll: *done = 1 when finished, then res is filled (caller arrays sized by
 * gf_server_nfree), plus submit-to-done latency in seconds. */
int gf_server_poll(gf_server* srv, uint64_t ticket, gf_fit_result* res, double* latency_s,
                   int* done);
int gf_server_nfree(gf_server* srv, uint64_t ticket, int* n);
/* Wait until every submitted fit has finished (bounded by wait_timeout_s per fit). */
int gf_server_drain(gf_server* srv);
/* Counters: ticks run, GPU launches made, peak slots in use. */
int gf_server_stats(gf_server* srv, int64_t* ticks, int64_t* launches, int* peak_slots);
int gf_server_destroy(gf_server* srv);

/* ---- introspection ----------------------------------------------------------------- */
/* Device-side time of the last evaluation's kernels (ms, CUDA events) and the number of
 * kernel launches it made. */
int gf_last_eval_stats(gf_ctx* ctx, double* kernel_ms, int* launches);
/* Device time (ms) of the last evaluation: all its kernels, and the final stream kernel
 * alone (the event pass, CUDA events on the context's stream). */
int gf_last_eval_times(gf_ctx* ctx, double* total_ms, double* stream_ms);
/* Whether the last evaluation replayed a captured CUDA graph (*replayed = 1) or launched
 * its kernels one by one (0: the first evaluation of a kind, one that had cache work to
 * do, or a context whose graph capture failed -- then why_not, if given, receives the
 * reason, at most n bytes with the terminating NUL; the context then launches directly
 * from there on, with the same results). */
int gf_last_eval_graph(gf_ctx* ctx, int* replayed, char* why_not, size_t n);
/* Allow (enable != 0, the default) or forbid the context to keep its own copy of a 1D
 * data set sorted ascending by the observable of the first Voigtian leaf.  Sorted, each
 * GPU thread takes a contiguous run of events and evaluates the Faddeeva function w(z)
 * once per run of 24, expanding it around that point for the others; the NLL is the same
 * sum (order-independent up to rounding) and gf_logpdf still returns log P_i in the
 * caller's event order.  The sort happens in gf_set_data (columns copied by the library
 * only, never gf_set_data_device), and again on the second evaluation after
 * gf_update_data; it costs one radix sort and 4 bytes per event for the permutation.
 * Takes effect at the next gf_set_data.  The fit server turns it off for its requests. */
int gf_set_event_sort(gf_ctx* ctx, int enable);
/* Evaluate a 1D tree that is an AddPdf of leaves (up to 4 components, each leaf with at
 * most 3 parameters) directly as P = sum_k c_k L_k with its gradient, and a single
 * exponential or Gaussian leaf, or a ProdPdf of up to 4 of them over at most two
 * observables (Listing 1, Listing 2), directly as log P = sum_k log L_k (enable != 0,
 * the default); or run both on the general postfix stack machine (0).  Both compute the
 * same quantities (Sec. 3's AddPdf and ProdPdf); the direct forms avoid the stack's
 * per-operation gradient vectors.  Takes effect at the next evaluation. */
int gf_set_mixture_path(gf_ctx* ctx, int enable);
/* Turn the replay of captured evaluation graphs on (enable != 0, the default) or off (every
 * evaluation launches its kernels one by one; the results are the same bits). */
int gf_set_graphs(gf_ctx* ctx, int enable);

/* ---- allocation-free evaluation -------------------------------------------------------
 * The paper has no counterpart to this call.  It is for callers that cannot call
 * cudaMalloc: code whose device memory is handed out by a pool or framework that grants
 * no extra buffers, or that must not grow the process's device footprint once running.
 * gf_nll_noalloc computes the same NLL as gf_nll for the 1D PDF tree rooted at `root` of
 * a context that holds only the model (gf_create and node declarations allocate no device
 * memory; no gf_set_data is needed), over caller-owned device columns, and allocates
 * nothing: its working buffers (theta, normalisation records, block partials, counters,
 * the compiled program) are one static device array of 440 KiB compiled into the library,
 * which every GPU that loads the library holds until the process exits.  The array is made
 * resident when the first context is created on a device (gf_create looks up its address
 * there), so the footprint does not grow at the first call.
 *   obs[k], dev_cols[k]: observable id and device column of n doubles (16-byte aligned);
 *   theta: host array of the free parameters (gf_free_params order);
 *   nll_dev: one double in device memory, written when the context's stream reaches it
 *            (the call returns after queueing; synchronise the stream before reading).
 * Limits: at most 256 parameters and 64 observables in the context, 24 free parameters,
 * 262,144 normalisation-grid bins in total, 32 instructions of the compiled tree; beyond
 * them, or for a node other than the exponential, Gaussian, Voigtian, threshold and
 * polynomial leaves, AddPdf and ProdPdf, the call returns GF_EINVAL with a message
 * (gf_last_error).
 * Each call looks up the array's device address (cudaGetSymbolAddress) with the context's
 * device current and stages theta and the compiled program from its own stack frame
 * (pageable host memory); it therefore returns GF_EINVAL, queueing nothing, while the
 * context's stream is capturing a graph.  Every call reuses the same array, which keeps
 * the last call's contents (the call clears what must start at zero): calls whose GPU
 * work overlaps -- other streams, other host threads -- race on it and must be
 * serialised by the caller. */
int gf_nll_noalloc(gf_ctx* ctx, int root, int nobs, const int* obs, int64_t n,
                   const double* const* dev_cols, const double* theta, double* nll_dev);

#ifdef __cplusplus
}
#endif
#endif /* GF_H */
