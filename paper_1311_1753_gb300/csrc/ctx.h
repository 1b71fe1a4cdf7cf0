// ctx.h -- the context object behind gf_ctx (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gf.h"
#include "gf_internal.h"
#include "launch.h"

namespace gfi {

enum NodeType { N_EXP = 1, N_GAUSS, N_VOIGT, N_THRESH, N_POLY, N_RELBW, N_ADD = 10, N_PROD,
                N_DALITZ, N_CONV, N_MAPPED, N_COMPOSITE, N_TDDP };

struct ObsDef {
  std::string name;
  double lo, hi;
};
struct ParDef {
  std::string name;
  double value, step, lo, hi;
  bool fixed;
};
struct NodeDef {
  int type;
  int obs = -1, obs2 = -1, obs3 = -1, obs4 = -1;  // N_TDDP: s12, s13, t, sigma_t
  std::vector<int> pars;      // leaf parameters / ADD fractions
  std::vector<int> children;  // ADD / PROD
  int nbx = 10000, nby = 0;   // normalisation grid (N_CONV: lattice bins, default 1000)
  int aux = 0;                // N_RELBW: orbital angular momentum
  gf_dalitz_kin kin{};
  std::vector<gf_resonance> res;
};

// Device state of a compiled tree + dataset.
struct DevState {
  // data
  int nobs = 0;
  int64_t n = 0;
  std::vector<int> obs_ids;           // dataset column k -> observable id
  std::vector<double*> cols;          // device columns
  bool owns_cols = false;
  // common
  double* theta = nullptr;            // all parameters (device)
  Program* prog = nullptr;            // compiled 1D program (device)
  double* derived = nullptr;
  float4* sbtab = nullptr;            // signal + background form: the table of w expansions
  double* partials = nullptr;
  double* partials2 = nullptr;
  unsigned* counters = nullptr;       // [0] events, [1] norm
  double* result = nullptr;           // [1 + nfree]: device mapping of h_result
  double* norm_out = nullptr;
  double* h_theta = nullptr;          // pinned
  double* h_result = nullptr;         // pinned
  size_t partials_cap = 0, partials2_cap = 0;
  int nblocks = 0;
  int nblocks_mixed = 0;              // signal + background form: the mixed plan's grid
  // Dalitz
  uint8_t* inside = nullptr;
  double* grid_cols = nullptr;
  double* gram = nullptr;
  void* ev_cache = nullptr;
  void* ev_cache64 = nullptr;           // FP64 per-event cache of a mixed context (refinement)
  float* fcols = nullptr;
  int* todo = nullptr;
  std::vector<double> ev_m0, ev_g0;     // shapes the event cache was built with (NaN: none)
  std::vector<double> ev64_m0, ev64_g0; // same for ev_cache64
  std::vector<double> col_m0, col_g0;   // shapes of the grid columns
  bool gram_valid = false;
  bool mask_built = false;
  // timing
  cudaGraphExec_t graph[24] = {};     // steady-state evaluation graphs: grad | fp64 << 1 |
                                      // direct << 2 | cur_set << 3
  bool graph_off = false;             // a capture failed: launch directly from then on
  std::string graph_why;              // why (for gf_last_eval_graph)
  void* tick_desc = nullptr;          // Fit1D / FitDz for batched ticks (device)
  int tick_kind = 0;                  // 0: none, 1: 1D, 2: Dalitz (Gram normalisation),
                                      // 3: 1D signal + background (FitSB after the Fit1D,
                                      // 256-byte aligned)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evm = nullptr;  // eval start, stream kernel, end
  int* flag = nullptr;                // data check (0 = ok): slot 63 of h_result, mapped
  // sorted layout of owned 1D columns (ascending by the first Voigtian's observable)
  bool sorted = false;
  int sort_obs = -1;                  // the column the events are sorted by
  int32_t* perm = nullptr;            // sorted position -> original event index
  int evals_since_load = 0;           // evaluations since the columns were (re)loaded
  // the next data sets prefetched by gf_prefetch_data (up to kStage in flight): copied and
  // range-checked in order on copy_stream into the spare buffer sets, swapped in by
  // gf_update_data; the graphs of each of the 1 + kStage buffer sets are kept (key cur_set)
  static constexpr int kStage = 2;
  std::vector<double*> stage[kStage];   // spare buffer sets (same sizes as cols)
  int stage_id[kStage] = {1, 2};        // their buffer-set numbers (cols has cur_set)
  cudaStream_t copy_stream = nullptr;
  cudaStream_t check_stream = nullptr;  // the range checks (off the copy stream: a check
                                        // waits for free SMs, the next copy need not)
  cudaEvent_t ev_copied[kStage] = {};   // recorded after each spare set's copy
  cudaEvent_t ev_staged[kStage] = {};   // ... and after its range check
  cudaEvent_t ev_free = nullptr;        // the compute stream's work before a copy
  std::vector<const double*> stage_src[kStage];  // host columns staged there (empty: none)
  int pend[kStage] = {0, 0};            // the spare sets holding prefetches, oldest first
  int npend = 0;
  int cur_set = 0;
  // convolution nodes: device descriptors and their tables (allocated at compile)
  std::vector<void*> conv_bufs;        // every allocation of the conv tables
  ConvDesc* conv_desc[kMaxConv] = {};  // device copies
  ConvDesc conv_host[kMaxConv] = {};
  int nconv = 0;
  // grid-normalised nodes (MappedPdf, CompositePdf)
  std::vector<void*> gn_bufs;
  GNormDesc* gn_desc[kMaxGNorm] = {};
  GNormDesc gn_host[kMaxGNorm] = {};
  int ngn = 0;
  // time-dependent Dalitz model: per-event amplitudes, grid columns, the three grid sums
  float4* tddp_cache = nullptr;  // per-event amplitudes as float pairs
  double2* tddp_gcols = nullptr;
  double2* tddp_gram = nullptr;
  bool tddp_ready = false;             // caches built for the loaded events
  float4* tddp_dcache = nullptr;       // free shapes: per-event shape derivatives
  double* tddp_normd = nullptr;        // free shapes: N and dN from the direct cell pass
  std::vector<double> tddp_shape;      // (m0, Gamma0) per resonance the cache was built with
  // binned data: bin contents and chi-squared variances (device), N x bin volume
  bool binned = false;
  double* bw = nullptr;
  double* bs2 = nullptr;
  double kbin = 0.0;
};

}  // namespace gfi

struct gf_dataset {
  gf_ctx* ctx;
  std::vector<int> obs;
  std::vector<std::vector<double>> cols;
  int64_t n = 0;
  // binned data set: cols hold the bin centres, w the contents, s2 the variances of the
  // chi-squared metric, kbin = (sum of contents) x (bin volume)
  bool binned = false;
  std::vector<double> w, s2;
  double kbin = 0.0;
};

struct gf_ctx {
  int device = 0;
  int precision = GF_FP64;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
  std::vector<gfi::ObsDef> obs;
  std::vector<gfi::ParDef> pars;
  std::vector<gfi::NodeDef> nodes;
  // compiled
  int root = -1;
  bool compiled = false;
  bool is_dalitz = false;
  bool is_tddp = false;      // time-dependent Dalitz model (Sec. 4's mixing fit)
  gfi::TddpPlan tplan{};
  bool has_grid = false;
  gfi::Program prog{};
  bool use_sb = false;       // the program is a signal + background AddPdf (k_sigbkg.cu)
  gfi::SigBkgDesc sb{};
  gfi::DalitzPlan dplan{};
  std::vector<int> free_ids;     // theta position -> parameter id
  std::vector<int> free_pos;     // parameter id -> theta position or -1
  gfi::DevState dev;
  int sm_count = 0;
  double last_ms = 0.0;
  double last_stream_ms = 0.0;
  int last_launches = 0;
  bool eval_in_flight = false;  // gf_nll_grad_start queued an evaluation, not yet finished
  bool eval_grad = false;       // ... with its gradient
  bool last_graph = false;  // the last evaluation replayed a captured graph
  bool graphs = true;       // replay captured graphs of steady evaluations
  bool event_sort = true;   // keep owned 1D columns sorted for the chunked event loop
  bool mixture_path = true; // evaluate AddPdf-of-leaves programs without the stack machine
  int metric = GF_METRIC_NLL; // the fit's metric over events or bins (gf_set_metric)
};

namespace gfi {
// capi.cpp internals used by fit.cpp and server.cpp
int set_error(gf_ctx* ctx, int code, const std::string& msg);
int ensure_compiled(gf_ctx* ctx);
// Evaluate at theta (free params): nll always, grad if non-null.  Blocking.
int evaluate(gf_ctx* ctx, const double* theta, double* nll, double* grad, bool fp64 = false);
// Enqueue an evaluation without waiting: the result lands in ctx->dev.h_result after the
// stream reaches it (used by the server to overlap fits).
int evaluate_async(gf_ctx* ctx, const double* theta, bool grad, bool fp64 = false);
int evaluate_finish(gf_ctx* ctx, double* nll, double* grad, bool grad_wanted);
size_t device_bytes_for(const gf_ctx* ctx, int root, int64_t n);
// Batched ticks: build the context's device descriptor once it has been evaluated (returns
// 0 if the context cannot join a batch: Dalitz with free shapes, or not evaluated yet);
// theta_all for theta; the 1 + nfree results of a batched evaluation checked as in
// evaluate_finish.
int tick_prepare(gf_ctx* ctx);
void fill_theta_all(const gf_ctx* ctx, const double* theta, double* out);
// the signal + background form: this theta_all's table layout (SBTabHdr) at
// theta_all + prog.rec_off; theta_all_size: the doubles a theta_all buffer then needs
void sbtab_fill(const gf_ctx* ctx, double* theta_all);
int theta_all_size(const gf_ctx* ctx);
int tick_finish(gf_ctx* ctx, const double* res, double* nll, double* grad);
int nfree(const gf_ctx* ctx);
const WeidCoef& weideman();
}  // namespace gfi
