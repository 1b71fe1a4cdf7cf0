// k_noalloc.cu -- gf_nll_noalloc: the 1D NLL over caller-owned device columns with no
// allocation at all.  Some callers cannot call cudaMalloc (their device memory belongs to
// a pool or framework that hands out no extra buffers, or they must not grow the
// process's footprint after start-up).  This entry point runs the same normalisation and
// event kernels as gf_nll, but every scratch buffer those kernels need (theta, leaf
// records, block partials, completion counters) lives in one file-scope static device
// array of fixed size.  The PDF tree is compiled on the host without heap allocation.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/gf.h"
#include "ctx.h"
#include "launch.h"

namespace gfi {
namespace {

// Limits of the static scratch (documented in gf.h).
constexpr int kNAMaxPar = 256;          // parameters of the context
constexpr int kNAMaxEvBlocks = 2048;    // event-kernel blocks (any n: the kernel strides)
constexpr int kNAMaxGridBlocks = 1024;  // normalisation blocks: <= 262,144 grid bins in total
constexpr int kNAStride = 1 + kMaxFree1D;
// Layout of the array, in doubles.
constexpr size_t kNATheta = 0;
constexpr size_t kNADerived = kNATheta + kNAMaxPar;
constexpr size_t kNAPartNorm = kNADerived + kMaxLeaf * kLeafRec + kMaxCoef;
constexpr size_t kNAPartEv = kNAPartNorm + (size_t)kNAMaxGridBlocks * 4;
constexpr size_t kNACounters = kNAPartEv + (size_t)kNAMaxEvBlocks * kNAStride;
constexpr size_t kNAProg = kNACounters + 2;  // two unsigned counters, one slot each
constexpr size_t kNADoubles = kNAProg + (sizeof(Program) + 7) / 8;

}  // namespace
}  // namespace gfi

// The scratch itself: one array per GPU that loads the library, alive until exit.
static __device__ __align__(256) double g_noalloc_scratch[gfi::kNADoubles];

namespace gfi {
namespace {

// Device address of the array in the current device's context.  Looked up on every call
// (cheap, allocation-free): a cached address would go stale after a device reset or
// under another context.
int scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return GF_ECUDA;
  }
  *out = static_cast<double*>(p);
  return GF_OK;
}

// Heap-free compile of a 1D tree into a postfix Program (same opcodes and order rules as
// the context compiler: Sethi-Ullman child order, log domain for exponential/Gaussian
// leaves and their products).
struct NACompiler {
  const gf_ctx* ctx;
  Program& P;
  const int* col_of_obs;  // observable id -> column, -1 if absent
  const int* free_pos;    // parameter id -> theta position, -1 if fixed
  const char* err = nullptr;
  int depth = 0, maxdepth = 0;

  int need(int id) const {
    const NodeDef& nd = ctx->nodes[id];
    if (nd.type != N_ADD && nd.type != N_PROD) return 1;
    int nn[kMaxLocal];
    const int nc = (int)nd.children.size();
    for (int k = 0; k < nc; ++k) nn[k] = need(nd.children[k]);
    for (int a = 1; a < nc; ++a)  // descending insertion sort
      for (int b = a; b > 0 && nn[b] > nn[b - 1]; --b) {
        const int t = nn[b]; nn[b] = nn[b - 1]; nn[b - 1] = t;
      }
    int m = 0;
    for (int k = 0; k < nc; ++k) m = nn[k] + (k > 0 ? 1 : 0) > m ? nn[k] + (k > 0 ? 1 : 0) : m;
    return m;
  }
  void order(const NodeDef& nd, int* idx) const {  // stable, by need, descending
    const int nc = (int)nd.children.size();
    int nn[kMaxLocal];
    for (int k = 0; k < nc; ++k) { idx[k] = k; nn[k] = need(nd.children[k]); }
    for (int a = 1; a < nc; ++a)
      for (int b = a; b > 0 && nn[idx[b]] > nn[idx[b - 1]]; --b) {
        const int t = idx[b]; idx[b] = idx[b - 1]; idx[b - 1] = t;
      }
  }
  bool emit(const Instr& I) {
    if (P.n >= kMaxIns) { err = "PDF tree too large (more than 32 instructions)"; return false; }
    P.ins[P.n++] = I;
    if (I.op == OP_LEAF) ++depth;
    if (I.op == OP_MUL || I.op == OP_LMUL || I.op == OP_ADD) --depth;
    if (depth > maxdepth) maxdepth = depth;
    return true;
  }
  bool natural_log(int id) const {
    const NodeDef& nd = ctx->nodes[id];
    if (nd.type == N_EXP || nd.type == N_GAUSS) return true;
    if (nd.type != N_PROD) return false;
    for (int c : nd.children)
      if (!natural_log(c)) return false;
    return true;
  }
  // returns 1 (log domain), 0 (linear) or -1 (error); *used gets the observable mask
  int walk(int id, uint64_t* used) {
    const NodeDef& nd = ctx->nodes[id];
    *used = 0;
    if (nd.type >= N_EXP && nd.type <= N_POLY) {
      if (P.nleaf >= kMaxLeaf) { err = "more than 16 leaves"; return -1; }
      if (nd.obs < 0 || nd.obs >= 64) { err = "observable id >= 64"; return -1; }
      const int col = col_of_obs[nd.obs];
      if (col < 0) { err = "no column for an observable used by the PDF"; return -1; }
      *used = 1ull << nd.obs;
      LeafDesc& L = P.leaf[P.nleaf];
      L = LeafDesc{};
      L.kind = nd.type;
      L.obs = col;
      L.npar = (int)nd.pars.size();
      for (int k = 0; k < L.npar; ++k) L.par[k] = nd.pars[k];
      L.nbins = (nd.type == N_VOIGT || nd.type == N_THRESH) ? nd.nbx : 0;
      L.lo = ctx->obs[nd.obs].lo;
      L.hi = ctx->obs[nd.obs].hi;
      Instr I{};
      I.op = OP_LEAF;
      I.kind = nd.type;
      I.obs = col;
      I.slot = P.nleaf;
      I.npar = L.npar;
      for (int k = 0; k < kMaxLocal; ++k) I.gidx[k] = k < L.npar ? free_pos[L.par[k]] : -1;
      ++P.nleaf;
      if (!emit(I)) return -1;
      return (nd.type == N_EXP || nd.type == N_GAUSS) ? 1 : 0;
    }
    if (nd.type != N_ADD && nd.type != N_PROD) {
      err = "unsupported node (exponential, Gaussian, Voigtian, threshold and polynomial "
            "leaves, AddPdf and ProdPdf only)";
      return -1;
    }
    const int nc = (int)nd.children.size();
    int idx[kMaxLocal];
    order(nd, idx);
    const bool prod = nd.type == N_PROD;
    const bool all_log = prod && natural_log(id);
    for (int k = 0; k < nc; ++k) {
      const int j = idx[k];
      uint64_t u = 0;
      const int d = walk(nd.children[j], &u);
      if (d < 0) return -1;
      if (prod && (u & *used)) { err = "ProdPdf factors share an observable"; return -1; }
      *used |= u;
      if (d == 1 && !all_log) {
        Instr T{};
        T.op = OP_TOLIN;
        if (!emit(T)) return -1;
      }
      if (!prod) {
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
        S.kind = C.sign;
        S.npar = C.n;
        for (int q = 0; q < kMaxLocal; ++q) S.gidx[q] = q < C.n ? free_pos[C.par[q]] : -1;
        ++P.ncoef;
        if (!emit(S)) return -1;
      }
      if (k > 0) {
        Instr M{};
        M.op = prod ? (all_log ? OP_LMUL : OP_MUL) : OP_ADD;
        if (!emit(M)) return -1;
      }
    }
    return all_log ? 1 : 0;
  }
};

bool acyclic(const gf_ctx* ctx, int id, int depth) {
  if (depth > 64) return false;
  for (int c : ctx->nodes[id].children)
    if (!acyclic(ctx, c, depth + 1)) return false;
  return true;
}

}  // namespace

// Called when a context is created on a device (that device current): the lookup loads
// this unit's module, so the array is resident from then on rather than appearing at the
// first gf_nll_noalloc call.
cudaError_t noalloc_preload() {
  void* p = nullptr;
  return cudaGetSymbolAddress(&p, g_noalloc_scratch);
}

}  // namespace gfi

using namespace gfi;

extern "C" int gf_nll_noalloc(gf_ctx* ctx, int root, int nobs, const int* obs, int64_t n,
                              const double* const* dev_cols, const double* theta,
                              double* nll_dev) {
  if (!ctx || !obs || !dev_cols || !nll_dev || n < 0 || nobs < 1 || nobs > kMaxObs)
    return GF_EINVAL;
  if (root < 0 || root >= (int)ctx->nodes.size())
    return set_error(ctx, GF_EINVAL, "gf_nll_noalloc: unknown root node");
  const int npar = (int)ctx->pars.size();
  if (npar > kNAMaxPar)
    return set_error(ctx, GF_EINVAL, "gf_nll_noalloc: more than 256 parameters in the context");
  if ((int)ctx->obs.size() > 64)
    return set_error(ctx, GF_EINVAL, "gf_nll_noalloc: more than 64 observables in the context");
  for (int k = 0; k < nobs; ++k) {
    if (obs[k] < 0 || obs[k] >= (int)ctx->obs.size() || !dev_cols[k])
      return set_error(ctx, GF_EINVAL, "gf_nll_noalloc: bad observable id or column");
    if (reinterpret_cast<uintptr_t>(dev_cols[k]) % 16 != 0)
      return set_error(ctx, GF_EINVAL, "gf_nll_noalloc: device columns must be 16-byte aligned");
  }
  if (!acyclic(ctx, root, 0)) return set_error(ctx, GF_EINVAL, "gf_nll_noalloc: cyclic tree");

  // parameter layout: theta_all on the stack, free positions in declaration order
  int free_pos[kNAMaxPar];
  double theta_all[kNAMaxPar];
  int nf = 0;
  for (int i = 0; i < npar; ++i) {
    theta_all[i] = ctx->pars[i].value;
    free_pos[i] = ctx->pars[i].fixed ? -1 : nf++;
  }
  if (nf > 0 && !theta)
    return set_error(ctx, GF_EINVAL, "gf_nll_noalloc: theta is NULL but parameters are free");
  if (nf > kMaxFree1D)
    return set_error(ctx, GF_EINVAL, "gf_nll_noalloc: more than 24 free parameters");
  for (int i = 0; i < npar; ++i)
    if (free_pos[i] >= 0) {
      if (!std::isfinite(theta[free_pos[i]]))
        return set_error(ctx, GF_EINVAL, "gf_nll_noalloc: non-finite theta");
      theta_all[i] = theta[free_pos[i]];
    }
  int col_of_obs[64];
  for (int o = 0; o < 64; ++o) col_of_obs[o] = -1;
  for (int k = 0; k < nobs; ++k) col_of_obs[obs[k]] = k;

  // compile (no heap): the Program lives on the stack
  Program P{};
  P.nobs = nobs;
  P.nfree = nf;
  P.tay_slot = -1;  // the caller's columns are used as they are: strided event loop
  P.sorted = 0;
  NACompiler C{ctx, P, col_of_obs, free_pos};
  uint64_t used = 0;
  const int dom = C.walk(root, &used);
  if (dom < 0) return set_error(ctx, GF_EINVAL, C.err);
  if (C.maxdepth > kMaxStack)
    return set_error(ctx, GF_EINVAL, "gf_nll_noalloc: PDF tree needs a deeper stack than 4");
  P.root_log = dom;
  int blk = 0;
  bool has_grid = false;
  for (int l = 0; l < P.nleaf; ++l) {
    LeafDesc& L = P.leaf[l];
    if (L.nbins > 0) {
      L.grid_first_block = blk;
      L.grid_nblocks = (L.nbins + kThreads - 1) / kThreads;
      blk += L.grid_nblocks;
      has_grid = true;
    }
  }
  P.ngrid_blocks = blk;
  if (blk > kNAMaxGridBlocks)
    return set_error(ctx, GF_EINVAL,
                     "gf_nll_noalloc: more than 262,144 normalisation-grid bins in total");

  // scratch: the static array's device address on this device
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return set_error(ctx, GF_ECUDA, "gf_nll_noalloc: cudaSetDevice failed");
  }
  cudaStream_t st = ctx->stream;
  // theta and the program are staged from this call's stack frame (pageable memory),
  // which a captured graph could not replay: refuse a capturing stream
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return set_error(ctx, GF_ECUDA, "gf_nll_noalloc: cudaStreamIsCapturing failed");
  }
  if (cap != cudaStreamCaptureStatusNone)
    return set_error(ctx, GF_EINVAL,
                     "gf_nll_noalloc: the context's stream is capturing; this call copies "
                     "theta and the program from host stack memory and cannot be captured");
  double* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return set_error(ctx, rc, "gf_nll_noalloc: cudaGetSymbolAddress failed");
  double* d_theta = base + kNATheta;
  double* d_derived = base + kNADerived;
  double* d_pnorm = base + kNAPartNorm;
  double* d_pev = base + kNAPartEv;
  unsigned* d_cnt_ev = reinterpret_cast<unsigned*>(base + kNACounters);
  unsigned* d_cnt_norm = reinterpret_cast<unsigned*>(base + kNACounters + 1);
  Program* d_prog = reinterpret_cast<Program*>(base + kNAProg);

  // event grid: same rule as the context path, capped by the scratch
  int per_sm = events_1d_blocks_per_sm(false, 0);
  per_sm = per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm);
  const int64_t want = ((n + 1) / 2 + kThreads1D - 1) / kThreads1D;
  int64_t nb = (int64_t)ctx->sm_count * per_sm;
  if (want < nb) nb = want;
  if (nb < 1) nb = 1;
  if (nb > kNAMaxEvBlocks) nb = kNAMaxEvBlocks;

  // theta from the caller's host array (staged by the runtime), counters cleared: the
  // array keeps the previous call's contents
  if (cudaMemcpyAsync(d_theta, theta_all, sizeof(double) * (npar > 0 ? npar : 1),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d_prog, &P, sizeof(Program), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(base + kNACounters, 0, 2 * sizeof(double), st) != cudaSuccess) {
    cudaGetLastError();
    return set_error(ctx, GF_ECUDA, "gf_nll_noalloc: queueing theta / program / counters failed");
  }
  const WeidCoef& W = weideman();
  cudaError_t e = cudaSuccess;
  if (has_grid) e = launch_norm_1d(P, d_prog, W, d_theta, d_pnorm, d_cnt_norm, d_derived, nullptr, nullptr, 0,
                                 st);
  Cols cols{};
  for (int k = 0; k < nobs; ++k) cols.c[k] = dev_cols[k];
  if (e == cudaSuccess)
    e = launch_events_1d(P, d_prog, W, cols, n, d_theta, d_derived, d_pev, d_cnt_ev, nll_dev,
                         nullptr, nullptr,
                         false, false, has_grid ? 0 : 1, (int)nb, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(ctx, GF_ECUDA, cudaGetErrorString(e));
  }
  return GF_OK;
}
