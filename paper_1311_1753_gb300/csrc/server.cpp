// server.cpp -- continuous-batching fit server (toy / pull studies).
//
// Requests (a model context + its events) queue on submit.  The scheduler admits a
// request when a slot is free and its device bytes fit in the memory budget, uploads its
// events (they stay resident until the fit ends) and starts a host thread that owns the
// fit's minimiser state.  Each minimiser step that needs NLL + gradient posts its theta
// and waits.  A scheduler "tick" takes every posted evaluation, enqueues all of them on
// the device back to back (each fit on its own stream, so their kernels overlap), then
// collects the results and wakes the fits.  Requests that arrive while others run are
// admitted at the next tick as slots and memory free up.  Every wait is bounded.
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/gf.h"
#include "ctx.h"
#include "fit.h"
#include "launch.h"

using namespace gfi;
using Clock = std::chrono::steady_clock;

namespace {

// normalisation-tick items (of kThreads threads) that build a signal + background fit's
// table of w expansions (its entries do not depend on how many threads build them)
constexpr int kTickTabItems = 64;

struct Req {
  uint64_t ticket = 0;
  gf_ctx* ctx = nullptr;
  gf_dataset* ds = nullptr;
  int root = -1;
  gf_fit_opts opts{};
  bool has_opts = false;
  size_t bytes = 0;
  Clock::time_point t_submit, t_done;
  // evaluation hand-off
  bool want = false, ready = false;
  bool want64 = false;  // FP64 evaluation (refinement stage of a mixed-precision fit)
  int evals = 0;        // evaluations done (the first one builds caches per fit)
  std::vector<double> theta, grad;
  double f = 0.0;
  int eval_rc = GF_OK;
  // outcome
  bool done = false;
  MinResult result;
  int nfree = 0;
  std::thread th;
};

}  // namespace

// Device and pinned buffers of the batched tick: the work lists of the four launches,
// every batched fit's theta_all, and their results.
struct TickBufs {
  int cap_fits = 0, cap_par = 0;
  TickItem* h_items = nullptr;  // [kLists][cap_fits]: 1D norm, 1D events (stack machine),
                                //   Dalitz events, signal + background events (the server's
                                //   precision), 1D events (AddPdf of leaves), 1D binned
                                //   events, signal + background events in FP64 (the
                                //   refinement steps of mixed fits)
  double* h_theta = nullptr;    // [cap_fits][cap_par]
  double* h_res = nullptr;      // [cap_fits][64]
  void* d_block = nullptr;      // device mirror of items + theta
  double* d_res = nullptr;
  cudaStream_t st = nullptr;
  static constexpr int kLists = 7;
  size_t bytes_items() const { return sizeof(TickItem) * kLists * cap_fits; }
  size_t bytes_theta() const { return sizeof(double) * (size_t)cap_fits * cap_par; }
};

struct gf_server {
  gf_server_opts opts{};
  TickBufs tb;
  int sm_count = 152;
  std::mutex mu;
  std::condition_variable cv_sched, cv_fit, cv_drain;
  std::deque<std::shared_ptr<Req>> pending;
  std::vector<std::shared_ptr<Req>> active;
  std::map<uint64_t, std::shared_ptr<Req>> all;
  std::atomic<bool> stop{false};
  std::thread sched;
  uint64_t next_ticket = 1;
  size_t used_bytes = 0;
  int64_t ticks = 0, launches = 0;
  int peak = 0;
  int64_t unfinished = 0;
};

// The root is an AddPdf of one Voigtian and one threshold leaf (the form k_sigbkg.cu
// evaluates; the compiler makes the final decision).
static bool sigbkg_form(const gf_ctx* ctx, int root) {
  if (root < 0 || root >= (int)ctx->nodes.size()) return false;
  const NodeDef& nd = ctx->nodes[root];
  if (nd.type != N_ADD || nd.children.size() != 2) return false;
  const int a = ctx->nodes[nd.children[0]].type, b = ctx->nodes[nd.children[1]].type;
  return (a == N_VOIGT && b == N_THRESH) || (a == N_THRESH && b == N_VOIGT);
}

static void fit_thread(gf_server* S, std::shared_ptr<Req> R) {
  const size_t n = R->ctx->free_ids.size();
  std::vector<double> x0(n), step(n), lo(n), hi(n);
  for (size_t k = 0; k < n; ++k) {
    const ParDef& p = R->ctx->pars[R->ctx->free_ids[k]];
    x0[k] = p.value;
    step[k] = p.step;
    lo[k] = p.lo;
    hi[k] = p.hi;
  }
  MinOpts mo;
  mo.up = R->ctx->metric == GF_METRIC_CHISQ ? 1.0 : 0.5;  // chi-squared: Delta chi2 = 1
  if (R->has_opts) {
    if (R->opts.tol > 0) mo.tol = R->opts.tol;
    if (R->opts.max_calls > 0) mo.max_calls = R->opts.max_calls;
    if (R->opts.up > 0) mo.up = R->opts.up;
    mo.hesse = R->opts.hesse != 0;
  }
  const double tmo = S->opts.wait_timeout_s > 0 ? S->opts.wait_timeout_s : 60.0;
  auto make_fg = [&](bool fp64) -> FGFun {
    return [&, fp64](const std::vector<double>& x, double& f, std::vector<double>& g) -> int {
    std::unique_lock<std::mutex> lk(S->mu);
    R->theta = x;
    R->want64 = fp64;
    R->want = true;
    R->ready = false;
    S->cv_sched.notify_all();
    if (!S->cv_fit.wait_for(lk, std::chrono::duration<double>(tmo),
                            [&] { return R->ready || S->stop.load(); }))
      return GF_ETIMEOUT;
    if (!R->ready) return GF_ETIMEOUT;
    f = R->f;
    g = R->grad;
    return R->eval_rc;
    };
  };
  const bool refine = R->ctx->precision == GF_MIXED && (R->ctx->is_dalitz || R->ctx->use_sb) &&
                      (!R->has_opts || R->opts.refine != 0);
  FGFun fg_fast = make_fg(false), fg_exact = make_fg(R->ctx->precision == GF_MIXED);
  MinResult m = refine ? minimise_refined(&fg_fast, fg_exact, x0, step, lo, hi, mo)
                       : minimise(fg_fast, x0, step, lo, hi, mo);
  std::lock_guard<std::mutex> lk(S->mu);
  R->result = std::move(m);
  R->nfree = (int)n;
  R->done = true;
  R->t_done = Clock::now();
  S->cv_sched.notify_all();
}

// One batched tick for fits with a tick descriptor: one host-to-device copy of the work
// lists and theta, the persistent launches (1D normalisation, 1D events, signal +
// background events, Dalitz events), one device-to-host copy of the results.  Returns the number of kernel launches.
static int64_t run_tick(gf_server* S, std::vector<std::shared_ptr<Req>>& fits) {
  TickBufs& T = S->tb;
  int maxpar = 1;
  for (auto& R : fits) maxpar = std::max(maxpar, theta_all_size(R->ctx));
  const int nfit = (int)fits.size();
  if (nfit > T.cap_fits || maxpar > T.cap_par) {  // (re)size the buffers
    if (T.st) cudaStreamSynchronize(T.st);
    cudaFreeHost(T.h_items);
    cudaFreeHost(T.h_theta);
    cudaFreeHost(T.h_res);
    cudaFree(T.d_block);
    cudaFree(T.d_res);
    T.cap_fits = std::max(nfit, std::max(T.cap_fits, S->opts.max_slots));
    T.cap_par = std::max(maxpar, std::max(T.cap_par, 64));
    if (cudaMallocHost(&T.h_items, T.bytes_items()) != cudaSuccess ||
        cudaMallocHost(&T.h_theta, T.bytes_theta()) != cudaSuccess ||
        cudaMallocHost(&T.h_res, sizeof(double) * 64 * T.cap_fits) != cudaSuccess ||
        cudaMalloc(&T.d_block, T.bytes_items() + T.bytes_theta()) != cudaSuccess ||
        cudaMalloc(&T.d_res, sizeof(double) * 64 * T.cap_fits) != cudaSuccess) {
      cudaGetLastError();
      for (auto& R : fits) R->eval_rc = GF_ENOMEM;
      T.cap_fits = T.cap_par = 0;
      return 0;
    }
  }
  if (!T.st) cudaStreamCreateWithFlags(&T.st, cudaStreamNonBlocking);
  TickItem* it_norm = T.h_items;
  TickItem* it_dz = T.h_items + 2 * T.cap_fits;
  TickItem* it_sb = T.h_items + 3 * T.cap_fits;
  TickItem* it_sb64 = T.h_items + 6 * T.cap_fits;
  int n_sb64 = 0, tot_sb64 = 0;
  // 1D event passes by mode (list 1: stack machine, 4: AddPdf of leaves, 5: binned)
  const int list1d[3] = {1, 4, 5};
  const int kind1d[3] = {kTick1DStack, kTick1DMixture, kTick1DBinned};
  int n1[3] = {0, 0, 0}, tot1[3] = {0, 0, 0};
  size_t smem1[3] = {0, 0, 0};  // the largest per-block scratch of each list's programs
  TickItem* d_items = static_cast<TickItem*>(T.d_block);
  double* d_theta = reinterpret_cast<double*>(static_cast<char*>(T.d_block) + T.bytes_items());
  int n_norm = 0, n_dz = 0, n_sb = 0, tot_norm = 0, tot_dz = 0, tot_sb = 0;
  int nfd = 0;
  for (int j = 0; j < nfit; ++j) {
    gf_ctx* c = fits[j]->ctx;
    fill_theta_all(c, fits[j]->theta.data(), T.h_theta + (size_t)j * T.cap_par);
    sbtab_fill(c, T.h_theta + (size_t)j * T.cap_par);
    const double* th = d_theta + (size_t)j * T.cap_par;
    double* res = T.d_res + 64 * j;
    if (c->dev.tick_kind == 1 || c->dev.tick_kind == 3) {
      if (c->has_grid) {
        // the signal + background form: kTickTabItems more items build its table
        const int ni = c->prog.ngrid_blocks + (c->dev.tick_kind == 3 ? kTickTabItems : 0);
        it_norm[n_norm++] = TickItem{c->dev.tick_desc, th, res, tot_norm, ni};
        tot_norm += ni;
      }
      if (c->dev.tick_kind == 3) {
        const void* fsb = static_cast<const char*>(c->dev.tick_desc) +
                          ((sizeof(Fit1D) + 255) / 256) * 256;
        // the grid of the plan the tick runs (the fit's standalone launches use the same);
        // a mixed fit's FP64 refinement steps run the FP64 plan in a list of their own
        const bool mixed = S->opts.precision == GF_MIXED && !fits[j]->want64;
        if (mixed) {
          it_sb[n_sb++] = TickItem{fsb, th, res, tot_sb, c->dev.nblocks_mixed};
          tot_sb += c->dev.nblocks_mixed;
        } else {
          it_sb64[n_sb64++] = TickItem{fsb, th, res, tot_sb64, c->dev.nblocks};
          tot_sb64 += c->dev.nblocks;
        }
      } else {
        const int m = c->prog.binned ? 2 : c->prog.mix ? 1 : 0;
        TickItem* it = T.h_items + (size_t)list1d[m] * T.cap_fits;
        it[n1[m]++] = TickItem{c->dev.tick_desc, th, res, tot1[m], c->dev.nblocks};
        tot1[m] += c->dev.nblocks;
        smem1[m] = std::max(smem1[m], events_1d_smem(c->prog, true, kThreads1D));
      }
    } else {
      it_dz[n_dz++] = TickItem{c->dev.tick_desc, th, res, tot_dz, c->dev.nblocks};
      tot_dz += c->dev.nblocks;
      nfd = std::max(nfd, (int)c->free_ids.size());
    }
  }
  cudaStream_t st = T.st;
  int64_t nl = 0;
  cudaError_t e = cudaMemcpyAsync(T.d_block, T.h_items, T.bytes_items() + 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_theta, T.h_theta, sizeof(double) * (size_t)nfit * T.cap_par,
                        cudaMemcpyHostToDevice, st);
  const WeidCoef& W = weideman();
  const int grid = S->sm_count * 4;
  if (e == cudaSuccess && n_norm) {
    e = launch_tick_1d(kTick1DNorm, d_items, n_norm, tot_norm, W, 0, grid, st);
    ++nl;
  }
  for (int m = 0; m < 3; ++m)
    if (e == cudaSuccess && n1[m]) {
      e = launch_tick_1d(kind1d[m], d_items + (size_t)list1d[m] * T.cap_fits, n1[m], tot1[m], W,
                         smem1[m], grid, st);
      ++nl;
    }
  if (e == cudaSuccess && n_sb) {
    e = launch_tick_sigbkg(true, d_items + 3 * T.cap_fits, n_sb, tot_sb, W, S->sm_count, st);
    ++nl;
  }
  if (e == cudaSuccess && n_sb64) {
    e = launch_tick_sigbkg(false, d_items + 6 * T.cap_fits, n_sb64, tot_sb64, W, S->sm_count,
                           st);
    ++nl;
  }
  if (e == cudaSuccess && n_dz) {
    const size_t smem = (size_t)nfd * kThreads * sizeof(double);
    e = launch_tick_dalitz(S->opts.precision == GF_MIXED, d_items + 2 * T.cap_fits, n_dz, tot_dz,
                           smem, S->sm_count * 2, st);
    ++nl;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(T.h_res, T.d_res, sizeof(double) * 64 * nfit, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (int j = 0; j < nfit; ++j) {
    auto& R = fits[j];
    R->grad.assign(R->ctx->free_ids.size(), 0.0);
    if (e != cudaSuccess) {
      R->eval_rc = GF_ECUDA;
      R->f = INFINITY;
    } else {
      R->eval_rc = tick_finish(R->ctx, T.h_res + 64 * j, &R->f, R->grad.data());
    }
    R->evals++;
  }
  if (e != cudaSuccess) cudaGetLastError();
  return nl;
}

static void scheduler(gf_server* S) {
  cudaSetDevice(S->opts.device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop.load()) {
    // retire finished fits: free their device memory and slot
    for (size_t i = 0; i < S->active.size();) {
      auto R = S->active[i];
      if (R->done) {
        lk.unlock();
        if (R->th.joinable()) R->th.join();
        gf_destroy(R->ctx);
        R->ctx = nullptr;
        gf_dataset_destroy(R->ds);
        R->ds = nullptr;
        lk.lock();
        S->used_bytes -= R->bytes;
        S->active.erase(S->active.begin() + i);
        S->unfinished--;
        S->cv_drain.notify_all();
      } else {
        ++i;
      }
    }
    // admit
    while (!S->pending.empty() && (int)S->active.size() < S->opts.max_slots) {
      auto R = S->pending.front();
      if (S->used_bytes + R->bytes > S->opts.mem_budget && !S->active.empty()) break;
      S->pending.pop_front();
      lk.unlock();
      // the batched 1D tick walks the events strided (a sorted copy would not pay for
      // itself), except for the signal + background form, whose tick takes each thread's
      // contiguous share of sorted events like the standalone kernel
      R->ctx->event_sort = sigbkg_form(R->ctx, R->root);
      int rc = gf_set_data(R->ctx, R->root, R->ds);
      // 1D fits: compiled and their tick descriptor prepared now, so that the first
      // evaluation joins the batched launches too
      if (rc == GF_OK && !R->ctx->is_dalitz && !R->ctx->is_tddp &&
          ensure_compiled(R->ctx) == GF_OK)
        tick_prepare(R->ctx);
      lk.lock();
      if (rc != GF_OK) {
        R->result.status = rc;
        R->done = true;
        R->t_done = Clock::now();
        S->unfinished--;
        S->cv_drain.notify_all();
        continue;
      }
      S->used_bytes += R->bytes;
      S->active.push_back(R);
      S->peak = std::max(S->peak, (int)S->active.size());
      R->th = std::thread(fit_thread, S, R);
    }
    // tick: every fit waiting for an evaluation
    std::vector<std::shared_ptr<Req>> batch;
    for (auto& R : S->active)
      if (R->want && !R->ready) batch.push_back(R);
    if (batch.empty()) {
      S->cv_sched.wait_for(lk, std::chrono::milliseconds(2));
      continue;
    }
    for (auto& R : batch) R->want = false;
    lk.unlock();
    int64_t nl = 0;
    // fits whose evaluation can join the batched launches: prepared (1D fits at
    // admission; Dalitz fits after their first evaluation, which builds the caches), and
    // not an FP64 refinement step unless the signal + background tick runs it
    std::vector<std::shared_ptr<Req>> batched, single;
    for (auto& R : batch) {
      const bool ready = R->ctx->dev.tick_desc && (R->evals > 0 || !R->ctx->is_dalitz);
      const bool plan = !R->want64 || R->ctx->dev.tick_kind == 3;
      if (ready && plan) batched.push_back(R);
      else single.push_back(R);
    }
    for (auto& R : single) {
      R->eval_rc = evaluate_async(R->ctx, R->theta.data(), true, R->want64);
      nl += R->ctx->last_launches;
    }
    if (!batched.empty()) nl += run_tick(S, batched);
    for (auto& R : single) {
      R->grad.assign(R->ctx->free_ids.size(), 0.0);
      if (R->eval_rc == GF_OK) R->eval_rc = evaluate_finish(R->ctx, &R->f, R->grad.data(), true);
      else R->f = INFINITY;
      R->evals++;
      if (!R->ctx->dev.tick_desc) tick_prepare(R->ctx);
    }
    lk.lock();
    S->ticks++;
    S->launches += nl;
    for (auto& R : batch) R->ready = true;
    S->cv_fit.notify_all();
  }
}

extern "C" {

int gf_server_create(const gf_server_opts* opts, gf_server** out) {
  if (!opts || !out || opts->max_slots < 1) return GF_EINVAL;
  gf_server* S = new gf_server();
  S->opts = *opts;
  cudaDeviceGetAttribute(&S->sm_count, cudaDevAttrMultiProcessorCount, opts->device);
  if (S->opts.wait_timeout_s <= 0) S->opts.wait_timeout_s = 60.0;
  S->sched = std::thread(scheduler, S);
  *out = S;
  return GF_OK;
}

int gf_server_submit(gf_server* S, gf_ctx* model, gf_dataset* ds, int root,
                     const gf_fit_opts* opts, uint64_t* ticket) {
  if (!S || !model || !ds || !ticket || ds->ctx != model) return GF_EINVAL;
  if (root < 0 || root >= (int)model->nodes.size()) return GF_EINVAL;
  if (model->precision != S->opts.precision) return GF_EINVAL;
  auto R = std::make_shared<Req>();
  R->ctx = model;
  R->ds = ds;
  R->root = root;
  if (opts) {
    R->opts = *opts;
    R->has_opts = true;
  }
  R->bytes = device_bytes_for(model, root, ds->n);
  R->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(S->mu);
  if (R->bytes > S->opts.mem_budget) return GF_ENOMEM;
  R->ticket = S->next_ticket++;
  *ticket = R->ticket;
  S->pending.push_back(R);
  S->all[R->ticket] = R;
  S->unfinished++;
  S->cv_sched.notify_all();
  return GF_OK;
}

int gf_server_nfree(gf_server* S, uint64_t ticket, int* n) {
  if (!S || !n) return GF_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return GF_EINVAL;
  auto& R = it->second;
  if (R->done) *n = R->nfree;
  else *n = R->ctx ? nfree(R->ctx) : 0;
  return GF_OK;
}

int gf_server_poll(gf_server* S, uint64_t ticket, gf_fit_result* res, double* latency_s,
                   int* done) {
  if (!S || !done) return GF_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return GF_EINVAL;
  auto& R = it->second;
  *done = R->done ? 1 : 0;
  if (!R->done) return GF_OK;
  const MinResult& m = R->result;
  if (res) {
    res->nll = m.fval;
    res->edm = m.edm;
    res->n_calls = m.calls;
    res->n_iter = m.iters;
    res->n_calls_fast = m.calls_fast;
    res->status = m.status;
    for (size_t k = 0; k < m.x.size(); ++k) {
      if (res->theta) res->theta[k] = m.x[k];
      if (res->err && k < m.err.size()) res->err[k] = m.err[k];
    }
    if (res->cov)
      for (size_t k = 0; k < m.cov.size(); ++k) res->cov[k] = m.cov[k];
  }
  if (latency_s)
    *latency_s = std::chrono::duration<double>(R->t_done - R->t_submit).count();
  return GF_OK;
}

int gf_server_drain(gf_server* S) {
  if (!S) return GF_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  const double tmo = S->opts.wait_timeout_s;
  while (S->unfinished > 0) {
    const int64_t before = S->unfinished;
    if (!S->cv_drain.wait_for(lk, std::chrono::duration<double>(tmo),
                              [&] { return S->unfinished < before || S->unfinished == 0; }))
      return GF_ETIMEOUT;
  }
  return GF_OK;
}

int gf_server_stats(gf_server* S, int64_t* ticks, int64_t* launches, int* peak_slots) {
  if (!S) return GF_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (ticks) *ticks = S->ticks;
  if (launches) *launches = S->launches;
  if (peak_slots) *peak_slots = S->peak;
  return GF_OK;
}

int gf_server_destroy(gf_server* S) {
  if (!S) return GF_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_sched.notify_all();
    S->cv_fit.notify_all();
  }
  if (S->sched.joinable()) S->sched.join();
  if (S->tb.st) cudaStreamSynchronize(S->tb.st);
  for (auto& kv : S->all) {
    auto& R = kv.second;
    if (R->th.joinable()) R->th.join();
    if (R->ctx) gf_destroy(R->ctx);
    if (R->ds) gf_dataset_destroy(R->ds);
    R->ctx = nullptr;
    R->ds = nullptr;
  }
  cudaFreeHost(S->tb.h_items);
  cudaFreeHost(S->tb.h_theta);
  cudaFreeHost(S->tb.h_res);
  cudaFree(S->tb.d_block);
  cudaFree(S->tb.d_res);
  if (S->tb.st) cudaStreamDestroy(S->tb.st);
  delete S;
  return GF_OK;
}

}  // extern "C"
