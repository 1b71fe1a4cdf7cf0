// launch.h -- host-side entry points of the kernel translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include "gf_internal.h"

namespace gfi {

// k_1d.cu
// P: the host copy (grid sizes); prog: the same program in device memory (read by the
// kernels, copied to shared memory per block)
// tab (or nullptr): the signal + background kernel's table of w expansions, built by
// tab_blocks extra blocks of the same launch from the header tab_hdr (device memory)
cudaError_t launch_norm_1d(const Program& P, const Program* prog, const WeidCoef& W,
                           const double* theta, double* partials, unsigned* counter,
                           double* derived, const SBTabHdr* tab_hdr, float4* tab,
                           int tab_blocks, cudaStream_t st);
size_t events_1d_smem(const Program& P, bool grad, int threads);
// store: out_logp[perm ? perm[i] : i] = log P_i (perm: the sort permutation of the
// data set, or nullptr); otherwise the NLL (and gradient) into result.
cudaError_t launch_events_1d(const Program& P, const Program* prog, const WeidCoef& W,
                             const Cols& cols, int64_t n,
                             const double* theta, const double* derived, double* partials,
                             unsigned* counter, double* result, double* out_logp,
                             const int32_t* perm, bool grad, bool store, int analytic_only,
                             int nblocks, cudaStream_t st);
// blocks per SM of the event kernel (mix: the AddPdf-of-leaves variant)
int events_1d_blocks_per_sm(bool grad, size_t smem, bool mix = false);
int events_logsum_blocks_per_sm(const Program& P);  // the direct log-sum kernel
// table uploads and kernel attributes, once per device (that device current)
cudaError_t prepare_kernels_1d();
// ConvolutionPdf tables of one node (after launch_norm_1d; before the event pass):
// host: the descriptor's sizes, dev: its device copy
cudaError_t launch_conv(const ConvDesc& host, const ConvDesc* dev, const WeidCoef& W, int nfree,
                        double* derived, cudaStream_t st);
// normalisation record of one grid-normalised node (after the convolutions)
cudaError_t launch_gnorm(const GNormDesc& host, const GNormDesc* dev, const WeidCoef& W,
                         int nfree, double* derived, cudaStream_t st);
// Sort (key, index) pairs ascending by the FP64 key (k_sort.cu): perm_tmp receives
// 0 .. n-1, perm_out the permutation, key_out the sorted keys.  temp == nullptr: only
// sets *temp_bytes to the scratch size the sort needs.
cudaError_t sort_by_key_f64(const double* key_in, double* key_out, int32_t* perm_tmp,
                            int32_t* perm_out, int64_t n, void* temp, size_t* temp_bytes,
                            cudaStream_t st);
// out[i] = in[perm[i]]
cudaError_t launch_gather(const double* in, const int32_t* perm, double* out, int64_t n,
                          cudaStream_t st);
cudaError_t prepare_kernels_dalitz();
// signal + background form (k_sigbkg.cu): NLL (+ gradient) into result[0 .. nfree], or
// with out_logp the per-event log P (through perm if sorted); mixed: the FP32 plan.  The
// kernel reads the sorted flag from the device copy of the program.  tab (or nullptr):
// the table of w expansions of this evaluation (header tab_hdr, ntab = 0: none), built
// by the normalisation launch before it.
cudaError_t launch_sigbkg(const SigBkgDesc& D, const WeidCoef& W, const Program* prog,
                          const double* x, int64_t n,
                          const double* derived, double* partials, unsigned* counter,
                          double* result, double* out_logp, const int32_t* perm, bool grad,
                          bool mixed, int nblocks, const SBTabHdr* tab_hdr, const float4* tab,
                          cudaStream_t st);
// host layout of the table (ntab = 0 when the line's cells would exceed kSBTabCap)
void sbtab_layout(double mu, double sigma, double gamma, double lo, double hi, SBTabHdr& H);
int sigbkg_blocks_per_sm(bool mixed);
// batched tick of signal + background fits (TickItem.fit -> FitSB)
// (grid: sm_count times the plan's resident blocks per SM)
cudaError_t launch_tick_sigbkg(bool mixed, const TickItem* items, int nfits, int total,
                               const WeidCoef& W, int sm_count, cudaStream_t st);
int sigbkg_threads(bool mixed);  // threads per block of the FP64 or the mixed plan
cudaError_t prepare_kernels_sigbkg();
// loads the allocation-free entry point's module (its static scratch array)
cudaError_t noalloc_preload();
// batched fit-server tick (persistent launches over a work list of TickItems)
// batched 1D ticks: the normalisation grids, or the event passes of one mode (the
// standalone kernel's: stack machine, AddPdf of leaves, binned)
constexpr int kTick1DNorm = 0, kTick1DStack = 1, kTick1DMixture = 2, kTick1DBinned = 3;
cudaError_t launch_tick_1d(int kind, const TickItem* items, int nfits, int total,
                           const WeidCoef& W, size_t smem, int grid, cudaStream_t st);
// flag := 1 if any event lies outside [lo[k], hi[k]] of its column
cudaError_t launch_check_range(const Cols& cols, int nobs, int64_t n, const double* lo,
                               const double* hi, int* flag, cudaStream_t st);

// k_dalitz.cu
struct DalitzBufs {
  const double* s12;
  const double* s13;
  const float* sf;          // FP32 plans: s12, s13, s23 as three float columns [3][n]
  int64_t n;
  const void* ev_cache;     // [ncached][n] double2 (FP64) or float2 (mixed)
  void* grid_cols;          // [nres + 1][nbx * nby] double2 (column 0 unused: a_NR = 1)
  const uint8_t* inside;    // [nbx * nby] cell-centre-inside mask
  double* gram;             // (nres + 1)^2 complex, interleaved
  double* norm_out;         // [1 + nfree]: N, dN/dtheta (direct norm pass)
  double* partials;         // per-block partials
  double* partials2;        // per-block partials of the norm pass
  unsigned* counter;
  unsigned* counter2;
  double* result;           // [1 + nfree]
  double* out_logp;         // per-event log P (store mode)
};
// mode flags for the event launch
enum DalitzNormMode { DN_GRAM = 0, DN_DIRECT = 1 };
cudaError_t launch_dalitz_mask(const DalitzPlan& D, uint8_t* inside, cudaStream_t st);
// flag := 1 if any event lies outside the kinematic region
cudaError_t launch_dalitz_check(const DalitzPlan& D, const double* s12, const double* s13,
                                int64_t n, int* flag, cudaStream_t st);
// FP32 columns s12, s13, s23 (s23 formed in FP64) for mixed-precision plans
cudaError_t launch_dalitz_fcols(const DalitzPlan& D, const double* s12, const double* s13,
                                int64_t n, float* fcols, cudaStream_t st);
cudaError_t launch_dalitz_ev_cache(const DalitzPlan& D, bool mixed, const double* theta,
                                   const double* s12, const double* s13, int64_t n,
                                   void* ev_cache, cudaStream_t st);
cudaError_t launch_dalitz_grid_cols(const DalitzPlan& D, const double* theta, const int* cols_todo,
                                    int ncols, void* grid_cols, const uint8_t* inside,
                                    cudaStream_t st);
cudaError_t launch_dalitz_gram(const DalitzPlan& D, const DalitzBufs& B, cudaStream_t st);
cudaError_t launch_dalitz_norm_direct(const DalitzPlan& D, bool mixed, bool grad,
                                      const double* theta, const DalitzBufs& B, int nblocks,
                                      cudaStream_t st);
cudaError_t launch_dalitz_events(const DalitzPlan& D, bool mixed, bool grad, bool store,
                                 int norm_mode, const double* theta, const DalitzBufs& B,
                                 int nblocks, cudaStream_t st);
int dalitz_blocks_per_sm(bool mixed, bool grad, bool cached_only, int nfree);
cudaError_t launch_tick_dalitz(bool mixed, const TickItem* items, int nfits, int total,
                               size_t smem, int grid, cudaStream_t st);
constexpr int kGramEntries = (kMaxRes + 1) * (kMaxRes + 2) / 2;

// time-dependent Dalitz model (k_dalitz.cu)
// per-event amplitudes a_r (at s12, s13) and b_r (at s12, s23): cache [2][nres][n], each
// complex value as two float pairs (re hi, re lo, im hi, im lo)
cudaError_t launch_tddp_cache(const TddpPlan& T, const double* theta, const double* s12,
                              const double* s13, int64_t n, float4* cache, cudaStream_t st);
// the three (nres+1)^2 complex grid sums G_A, G_B, X (dA sum conj(a_r) a_s, conj(b_r) b_s,
// conj(a_r) b_s; index 0 the non-resonant 1) into gram [3][(nres+1)^2]; gcols: scratch
// [2][nres][nbx nby] double2; inside: the cell mask
cudaError_t launch_tddp_gram(const TddpPlan& T, const double* theta, const uint8_t* inside,
                             double2* gcols, double2* gram, cudaStream_t st);
// NLL (+ gradient) into result[0 .. nfree], or (out_logp) per-event log P; nblocks at most
// kTddpBlocksPerSm x the SM count (all blocks resident, each a contiguous equal share of events)
constexpr int kTddpBlocksPerSm = 3;
cudaError_t launch_tddp_events(const TddpPlan& T, bool grad, const double* theta,
                               const double* const* cols, int64_t n, const float4* cache,
                               const float4* dcache, const double2* gram, const double* normd,
                               double* nscratch, double* partials, unsigned* counter,
                               double* result, double* out_logp, int nblocks, const WeidCoef& W,
                               cudaStream_t st);
// free resonance shapes: amplitudes and shape derivatives per event (dcache: 4 nres n), and
// N with dN/dtheta by a direct pass over the cells (out[0], out[1 + k])
cudaError_t launch_tddp_cache_free(const TddpPlan& T, const double* theta, const double* s12,
                                   const double* s13, int64_t n, float4* cache, float4* dcache,
                                   cudaStream_t st);
cudaError_t launch_tddp_norm_direct(const TddpPlan& T, const double* theta,
                                    const uint8_t* inside, double* partials, unsigned* counter,
                                    double* out, int nblocks, cudaStream_t st);

}  // namespace gfi
