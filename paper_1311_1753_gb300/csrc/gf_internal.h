// gf_internal.h -- plans shared by the host-side PDF-tree compiler (capi.cpp) and the
// sm_103a kernels (k_1d.cu, k_dalitz.cu).  Plain structs: the Dalitz plan and the
// Faddeeva table go to kernels by value (constant bank), the 1D program lives in device
// memory and each block copies it to shared memory.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gfi {

constexpr int kMaxIns = 32;     // instructions of a 1D program
constexpr int kMaxObs = 8;      // observables of one dataset
constexpr int kMaxLeaf = 16;    // leaves of a 1D program
constexpr int kMaxCoef = 16;    // fraction coefficients of a 1D program
constexpr int kMaxLocal = 8;    // parameters of one leaf
constexpr int kLeafRec = 20;    // doubles per leaf record: invN, logN, dlogN[8], c[10]
constexpr int kMaxFree1D = 24;  // free parameters of a 1D model with gradient
constexpr int kMaxStack = 4;    // evaluation stack depth (Sethi-Ullman ordered)
constexpr int kMaxRes = 12;     // resonances of a Dalitz model
constexpr int kWeidN = 40;      // terms of the Faddeeva series
constexpr int kThreads = 256;   // threads per block of the Dalitz and normalisation kernels
constexpr int kThreads1D = 128; // threads per block of the 1D event kernel (its gradient
                                // stack: 5 x nfree x 128 doubles of shared memory <= 123 KB)
constexpr int kMixMax = 4;      // components of an AddPdf evaluated without the stack machine
constexpr int kMixLocal = 3;    // ... each leaf with at most 3 local parameters
constexpr int kLogLeaf = 4;    // leaves of a log-domain product evaluated directly
constexpr int kChunk = 24;      // sorted 1D data: events per expansion of w (k_1d.cu); the
                                // chunked loop runs when there are >= kChunk/2 events per thread

// Leaf kinds (shape functions; Sec. 2-3 of the paper and gf.h).
enum Leaf : int32_t {
  L_EXP = 1, L_GAUSS = 2, L_VOIGT = 3, L_THRESH = 4, L_POLY = 5,
  L_RELBW = 6,  // relativistic Breit-Wigner line shape (grid-normalised)
  L_CONV = 7,   // a ConvolutionPdf read from its lattice table (k_conv_sum builds it)
  L_IND = 8,    // indicator of an interval of the observable (MappedPdf)
  L_GNORM = 9   // record of a grid-normalised node (MappedPdf, CompositePdf; k_gnorm)
};
constexpr int kRawLeaf = 0x100;  // LeafDesc.aux flag: the unnormalised shape (N = 1)
constexpr int kMaxGNorm = 2;     // grid-normalised nodes of one tree
constexpr int kResidCol = 7;     // observable column of a resolution's residual variable
constexpr int kMaxConv = 2;      // convolution nodes of one tree
constexpr int kConvMaxLattice = 65536;  // lattice bins of one convolution
constexpr int kConvMaxOffsets = 8193;   // resolution offsets of one convolution

// Opcodes of the postfix (stack) program of a 1D PDF tree.  "log" values live in the
// log domain, "lin" values in the linear domain; the compiler inserts TOLIN where a
// linear consumer needs a log value.
enum Op : int32_t {
  OP_LEAF = 1,    // push the normalised leaf value (log domain for EXP/GAUSS)
  OP_TOLIN = 2,   // s0 = exp(s0)
  OP_MUL = 3,     // s0 = s1 * s0        (ProdPdf, linear)
  OP_LMUL = 4,    // s0 = s1 + s0        (ProdPdf, log domain)
  OP_SCALE = 5,   // s0 = coef[slot] * s0 (AddPdf fraction, or 1 - sum of fractions)
  OP_ADD = 6,     // s0 = s1 + s0        (AddPdf)
  OP_COMPOSE = 7, // s0 = shell(s0): the shell leaf (slot, kind) of a CompositePdf
  OP_GNORM = 8,   // s0 = s0 / N of a grid-normalised node (record slot)
};

struct Instr {
  int32_t op;
  int32_t kind;              // OP_LEAF: Leaf kind; OP_SCALE: +1 (coef = f) / -1 (1 - sum f)
  int32_t obs;               // OP_LEAF: observable column
  int32_t slot;              // OP_LEAF: leaf record; OP_SCALE: coefficient slot
  int32_t npar;              // OP_LEAF: local parameters; OP_SCALE: fractions involved
  int32_t gidx[kMaxLocal];   // free index (theta position) of each, -1 when fixed
};

struct LeafDesc {
  int32_t kind, obs, npar, nbins;  // nbins > 0: midpoint-grid normalisation
  int32_t par[kMaxLocal];          // indices into theta_all
  double lo, hi;                   // observable range
  int32_t grid_first_block;        // first block of this leaf in the norm grid launch
  int32_t grid_nblocks;
  int32_t aux;                     // L_RELBW: orbital angular momentum; L_CONV: conv index
  int32_t pad;
};

struct CoefDesc {
  int32_t sign, n;                 // sign +1: coef = theta[par[0]]; -1: 1 - sum theta[par[k]]
  int32_t par[kMaxLocal];
};

struct Program {
  int32_t n, nleaf, ncoef, nfree, nobs, root_log, ngrid_blocks;
  int32_t tay_slot;  // leaf record of the first Voigtian leaf (expanded per chunk), -1: none
  int32_t tay_obs;   // its observable column
  int32_t sorted;    // events sorted ascending by column tay_obs (chunked event loop)
  // AddPdf of leaves (the program is K x [LEAF, (TOLIN), SCALE, (ADD)]): evaluated as
  // P = sum_k c_k L_k without the stack machine.  mix = K (2..kMixMax), 0: not a mixture.
  int32_t mix;
  int32_t mix_leaf[4], mix_log[4], mix_scale[4];  // instruction indices; TOLIN present
  // log-domain product of exponential and Gaussian leaves (the program is LEAF, then
  // K - 1 x [LEAF, LMUL], K <= kLogLeaf, at most 2 observables): log P = sum_k l_k is
  // evaluated directly, without the stack machine.  1: this form, 0: not.
  int32_t logsum;
  // log-sum programs: the leaves' records (kLogLeaf x kLeafRec doubles), then the same as
  // float pairs, computed on the host with theta and uploaded behind it at theta + rec_off;
  // the signal + background form: its table layout (SBTabHdr) there
  int32_t rec_off;
  // binned data (the events are bin centres): the metric over bins and its inputs.
  // binned = 0: unbinned events, metric -sum log P.
  int32_t binned, metric;  // metric: GF_METRIC_NLL / _BINNED_NLL / _CHISQ (gf.h)
  double kbin, logk;       // N x bin volume and its log: nu_b = kbin P(x_b)
  const double* bw;        // bin contents (device)
  const double* bs2;       // chi-squared variances (device)
  Instr ins[kMaxIns];
  LeafDesc leaf[kMaxLeaf];
  CoefDesc coef[kMaxCoef];
};

struct Cols {
  const double* c[kMaxObs];
};

// An AddPdf of one Voigtian and one threshold leaf over the same observable (either order;
// Sec. 4's line-shape fit), evaluated by k_sigbkg.cu: leaf-record and coefficient slots,
// the theta positions of the leaves' parameters (-1 when fixed) and of the fraction.
struct SigBkgDesc {
  int32_t slot_v, slot_t;    // leaf records (Voigtian, threshold)
  int32_t cslot_v, cslot_t;  // coefficient slots
  int32_t gv[3];             // mu, sigma, Gamma
  int32_t gt[3];             // x0, power, c
  int32_t fpos_v, fpos_t;    // the fraction in each coefficient
  int32_t fsgn_v, fsgn_t;    // +1: coefficient = f; -1: 1 - f
  int32_t nfree;
};

// The table of expansions of w along the line Im z = y of one evaluation (the signal +
// background kernel's Voigtian): entry j holds the degree-5 Taylor coefficients of w
// around z_j + i y, z_j the middle of cell j of Re z.  Cells: nneg logarithmic cells below
// -zc, ncore cells of width h from a, then logarithmic cells above zc (ratio e^lr), so
// that every cell's half-width stays within the expansion's validated limit.  The host
// lays the table out from theta (ntab = 0: no table this evaluation) and uploads this
// header with theta; the normalisation launch builds the entries.
struct SBTabHdr {
  int32_t ntab, nneg, ncore, pad0;
  float a, ih, h, zc, izc, ilr, lr, pad1;
  double mu, c1, ic1, y;  // Re z = (x - mu) c1, ic1 = 1/c1
};
constexpr int kSBTabCap = 1 << 15;  // entries, at most (2.6 MB)
constexpr int kSBTabF4 = 5;         // float4 per entry

// One grid-normalised node (MappedPdf, CompositePdf): N = h sum_b F(lo + (b + 1/2) h) over
// nbins midpoints of the observable, F the node's body (sub-program), with dN over the
// node's local parameters; k_gnorm writes the record at slot.
struct GNormDesc {
  const Program* sub;
  double* partials;  // [blocks][1 + kMaxLocal]
  unsigned* counter;
  int32_t nbins, slot, mcol, nloc;
  int32_t loc2free[kMaxLocal];
  double lo, h;
};

// One ConvolutionPdf node (k_1d.cu: k_conv_points, k_conv_sum).  Lattice x_i = lo + i h (i = 0..L); resolution
// offsets u_k = (kmin + k) h (k < K); model points t_j = lo + (j - kmax) h (j < J =
// L + K); C_i = h sum_k R(u_k) M(x_i - u_k).  Tables hold a value row, then one row per
// local parameter (the free parameters of the model and resolution subtrees).
struct ConvDesc {
  const Program* pm;  // model subtree as a program (device), its leaves in the main table
  const Program* pr;  // resolution subtree (its observable in column kResidCol)
  float2* mt;         // [1 + nloc][J] pairs (hi, lo)
  float2* rt;         // [1 + nloc][K]
  double* ct;         // [1 + nloc][L + 1]: C_i and dC_i/dtheta_l
  double* partials;   // [L + 1][1 + nloc]: trapezoid terms
  unsigned* counter;
  int32_t L, kmin, kmax, J, K, nloc;
  int32_t slot;        // leaf record of the conv leaf in the main program
  int32_t mcol;        // the model's observable column
  int32_t loc2free[kMaxLocal];
  double lo, h;
};

// Faddeeva coefficients (Weideman 1994 rational series) as double-float pairs, filled on
// the host.  Kept small: it is a kernel parameter.
struct WeidCoef {
  float Lhi, Llo;                           // L as a double-float pair
  float ahi[kWeidN + 1], alo[kWeidN + 1];   // a_n = ahi + alo
};

// ---- Dalitz plan ------------------------------------------------------------------
struct DalitzChannel {
  double ma2, mb2, mc2;  // squared masses of a, b (resonance pair) and bachelor c
  double thrA, thrB;     // (ma+mb)^2, (ma-mb)^2
  double k1;             // (M^2 - mc^2)(ma^2 - mb^2)          (Zemach S_1 constant)
  double a2c, a2k;       // a2 = s - a2c + a2k/s, a2c = 2M^2 + 2mc^2, a2k = (M^2-mc^2)^2
};

struct DalitzRes {
  int32_t channel, spin;
  int32_t p_m0, p_g0, p_re, p_im;  // theta_all indices
  int32_t g_m0, g_g0, g_re, g_im;  // free indices or -1
  int32_t ev_cached;               // per-event amplitude column available (cache slot or -1)
  int32_t grid_col;                // grid column index (always r + 1; 0 is a_NR)
};

struct DalitzPlan {
  double M2, sum_m2;  // M^2 and M^2 + m1^2 + m2^2 + m3^2
  double R2;          // Blatt-Weisskopf radius squared
  double m1, m2, m3, M;
  DalitzChannel ch[3];
  int32_t nres, nfree, nbx, nby;
  double x0, hx, y0, hy;  // grid: s12 = x0 + (i + 1/2) hx, s13 = y0 + (j + 1/2) hy
  DalitzRes res[kMaxRes];
};

// ---- time-dependent Dalitz model (Sec. 4: the mixing fit) -------------------------------
// The Dalitz plan (fixed resonance shapes) plus the time parameters: tau, mixing x, y and
// the resolution scale s (sigma = s sigma_t per event); theta_all indices and free
// indices (-1: fixed).  Data columns: s12, s13, t, sigma_t.
struct TddpPlan {
  DalitzPlan D;
  int32_t p_tau, p_x, p_y, p_s;
  int32_t g_tau, g_x, g_y, g_s;
  int32_t nfree;
  int32_t shape_free;        // some resonance mass or width is free: amplitudes and their
                             // shape derivatives per evaluation, N by a direct cell pass
  // the sigma_t density (dens = 1): Gamma(2) truncated to [slo, shi] with rate
  // exp(b0 + b1 (s12 - sc) + b2 (s13 - sc))
  int32_t dens;
  int32_t p_b0, p_b1, p_b2, g_b0, g_b1, g_b2;
  int32_t pad;
  double slo, shi, sc;
};

// ---- batched evaluation of many fits (one fit-server tick) ----------------------------
// Per-fit descriptors live in device memory; a tick's work list holds one TickItem per fit
// per launch: items item0 .. item0 + nitems - 1 of the launch are that fit's virtual
// blocks 0 .. nitems - 1, which process exactly the events of the fit's standalone
// blocks, so its result is the same bits alone or in the batch.
struct Fit1D {
  Program P;
  Cols cols;
  int64_t n;
  double* derived;
  double* partials;
  double* partials_norm;
  unsigned* counter_ev;
  unsigned* counter_norm;
  float4* sbtab;  // signal + background form: its table of w expansions (else nullptr)
  int analytic_only;
  int pad;
};

struct FitDz {
  DalitzPlan D;
  const double* s12;
  const double* s13;
  const float* sf;
  int64_t n;
  const void* ev_cache;
  const double* gram;
  double* partials;
  unsigned* counter;      // [0] arrivals, [2] the first block done (it forms N)
  double* norm_scratch;   // 1 + nfree doubles: N and dN/dtheta from that block
  int cache_wide;
  int pad;
};

// A signal + background fit in the batched tick (k_sigbkg.cu).
struct FitSB {
  SigBkgDesc D;
  const double* x;
  int64_t n;
  double* derived;
  double* partials;
  unsigned* counter;
  const float4* sbtab;  // the table of w expansions (layout at theta + rec_off)
  int32_t sorted;
  int32_t rec_off;
};

struct TickItem {
  const void* fit;       // Fit1D* or FitDz* (device)
  const double* theta;   // this fit's theta_all for this tick (device)
  double* result;        // its 1 + nfree results (device)
  int item0;             // first item of this fit in the launch
  int nitems;            // its virtual grid
};

}  // namespace gfi
