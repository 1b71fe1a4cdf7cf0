#!/usr/bin/env python
"""Benchmark of the unbinned-likelihood hot path on GB300.

Headline workload (default): the 1D composite fit (Voigtian + threshold background on
the D*+ - D0 mass-difference range, 10^7 FP64 events, 5 free parameters, 2 x 10,000-bin
normalisation grids).  One step = one NLL + gradient evaluation (theta upload, grid
normalisation, event pass with the fused gradient, deterministic reduction, result
download), as a minimiser call makes it.  Metric: events x evaluations per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload voigt|exp|dalitz|dalitz-mixed] [--no-extra] [--fits] [--serve]

N > 1 runs under torchrun: every rank evaluates its own data set (independent problems,
weak scaling, no data-path collective); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1311_1753_gb300 import synth  # noqa: E402

# Peaks: HBM from the driver's measurement; FP64 from the unit counts and the maximum
# clock (152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz); FP32 likewise (x 128).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

# The FP64 plans compute FP64-accurate results in double-float arithmetic (pairs of
# floats) on the FP32 pipe.  Each timed event kernel's FP32 flops per event (FADD + FMUL
# + 2 FFMA executed per event, predicated-on) and the DRAM traffic of one launch are ncu
# counters of one launch of this build at the bench's own size (the profile summaries
# of k_sigbkg and k_dalitz_stream under profiles/).
FP32_FLOPS_PER_EVENT = {"voigt_grad": 593.1,      # FADD 334.5 + FMUL 45.1 + 2 x FFMA 106.8
                        "voigt_grad_mixed": 104.6,  # FADD 38.3 + FMUL 18.2 + 2 x FFMA 24.0
                        "dalitz_cached": 1350.2,  # FADD 782.2 + FMUL 82.0 + 2 x FFMA 243.0
                        "dalitz_free": 7446.6,    # FADD 3933.6 + FMUL 531.0 + 2 x FFMA 1491.0
                        "dalitz_mixed": 902.1}    # FADD 204.1 + FMUL 280.0 + 2 x FFMA 209.0
TRAFFIC_PER_LAUNCH = {"voigt_grad": 81.85e6,        # 80.15 MB read + 1.70 MB written
                      "voigt_grad_mixed": 83.61e6,  # 80.47 MB read + 3.14 MB written
                      "dalitz_cached": 131.37e6,    # 128.14 MB read + 3.23 MB written (10^6)
                      "dalitz_free": 864.78e6,      # 164.37 MB read + 700.41 MB written (5 x 10^6;
                                                    # the writes are register spills)
                      "dalitz_mixed": 103.00e6}     # 100.10 MB read + 2.90 MB written (5 x 10^6)
# the headline workload's name, shared by both arms' JSON lines
VOIGT_WORKLOAD = ("1D composite: Voigtian (mu,sigma,Gamma) + threshold (c) with fraction f, "
                  "10^7 FP64 events, 2 x 10,000-bin grid normalisation")
# The method's work: the same pass in FP64 operations (FMA = 2, add/mul = 1, each exp,
# log, sqrt or division = 1), a fixed count (it does not follow the kernel's chunk length):
# w(z) by one Weideman series (N = 40: 305) and a degree-5 expansion amortised over 24
# events (recurrence ~40 per expansion, evaluation 20, argument 3) = 37 per event; Voigt
# value and 3 partials 31; threshold value and partial 9; the mixture (2 products, 1 sum)
# and its gradient terms (6 products, 6 sums) 15; log P and 1/P 2.
FP64_FLOPS_PER_EVENT = {"voigt_grad": 94}
# The free-shape Dalitz model (8 resonances, 7 with free mass and width, 30 free
# parameters), the method's FP64 operations per event counted the same way from the
# amplitude code: the kinematics of
# the 3 channels 95 (1/sqrt(s), break-up momentum, Blatt-Weisskopf factors, Zemach terms),
# 7 Breit-Wigner amplitudes 105 (running width, complex reciprocal, barrier and angular
# factors), 8 coefficient multiply-adds 64, |A|^2 and log 5; the gradient: 16 coefficient
# terms 82, 14 mass and width derivatives 273: 624.
FP64_FLOPS_PER_EVENT["dalitz_free"] = 624
# The fixed-shape Dalitz model: the pass reads each event's 8 cached amplitudes, FP64-
# accurate as float pairs (16 B each): 128 B/event from HBM.
BYTES_PER_EVENT = {"dalitz_cached": 128}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling during the timed region: every 100 ms, started before the region
    (its first line marks that the sampler runs); lines written before the region are
    left out of the summary when the region has lines of its own."""

    def __init__(self, index=0):
        self.path = tempfile.mktemp(suffix=".csv")
        self.n0 = 0
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader",
                                       "-i", str(index), "-lms", "100"],
                                      stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
            return
        t_end = time.perf_counter() + 3.0
        while time.perf_counter() < t_end and self.p.poll() is None:
            n = self._lines()
            if n > 0:
                self.n0 = n
                break
            time.sleep(0.02)

    def _lines(self):
        try:
            with open(self.path) as fh:
                return sum(1 for line in fh if line.count(",") >= 8)
        except OSError:
            return 0

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if len(rows) > self.n0:
            rows = rows[self.n0:]
        if not rows:
            return None
        sm = [float(r[1].split()[0]) for r in rows if r[1].split()[0].replace(".", "").isdigit()]
        mx = [float(r[2].split()[0]) for r in rows if r[2].split()[0].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---- workloads ------------------------------------------------------------------------------
def voigt_workload(gf, n, seed, precision):
    lo, hi = synth.VOIGT_RANGE
    x = synth.voigt_threshold_events(n, **synth.VOIGT_TRUTH, lo=lo, hi=hi, seed=seed)
    t = synth.VOIGT_TRUTH
    ctx = gf.Context(0, precision)
    xo = ctx.observable("dm", lo, hi)
    mu = ctx.parameter("mu", t["mu"], 1e-5, 0.143, 0.148)
    s = ctx.parameter("sigma", t["sigma"], 1e-5, 1e-5, 2e-3)
    w = ctx.parameter("width", t["width"], 1e-5, 1e-6, 1e-3)
    x0 = ctx.parameter("x0", t["x0"], 1e-4, fixed=True)
    pw = ctx.parameter("power", t["power"], 0.01, fixed=True)
    c = ctx.parameter("c", t["c"], 0.5, 0.0, 200.0)
    f = ctx.parameter("frac", t["frac"], 0.01, 0.0, 1.0)
    root = ctx.add([ctx.voigt(xo, mu, s, w), ctx.threshold(xo, x0, pw, c)], [f])
    ctx.set_data(root, [xo], [x])
    theta = np.array([t["mu"], t["sigma"], t["width"], t["c"], t["frac"]])
    return ctx, root, [xo], [x], theta


def exp_workload(gf, n, seed, precision):
    x = synth.exp_events(n, -1.0, seed=seed)
    ctx = gf.Context(0, precision)
    xo = ctx.observable("x", 0.0, 10.0)
    a = ctx.parameter("alpha", -2.0, 0.1, -10.0, 10.0)
    root = ctx.exp(xo, a)
    ctx.set_data(root, [xo], [x])
    return ctx, root, [xo], [x], np.array([-1.0])


def dalitz_spec():
    with open(os.path.join(ROOT, "tests", "golden", f"dalitz_model_{synth.SEED_DALITZ_MODEL}.json")) as fh:
        return json.load(fh)


def dalitz_context(gf, spec, precision, free_shapes):
    ctx = gf.Context(0, precision)
    o12 = ctx.observable("s12", 0.0, 4.0)
    o13 = ctx.observable("s13", 0.0, 4.0)
    res, theta = [], []
    nres = len(spec["resonances"])
    for i, r in enumerate(spec["resonances"]):
        shape_free = free_shapes and i != nres - 1
        m0 = ctx.parameter(f"m0_{i}", r["m0"], 0.005, 0.4, 1.75, fixed=not shape_free)
        g0 = ctx.parameter(f"g0_{i}", r["g0"], 0.005, 0.01, 0.6, fixed=not shape_free)
        re = ctx.parameter(f"re_{i}", r["re"], 0.01)
        im = ctx.parameter(f"im_{i}", r["im"], 0.01)
        res.append(dict(channel=r["channel"], spin=r["spin"], mass=m0, width=g0, re=re, im=im))
        theta += ([r["m0"], r["g0"]] if shape_free else []) + [r["re"], r["im"]]
    root = ctx.dalitz(o12, o13, spec["kin"], res)
    return ctx, root, [o12, o13], np.array(theta)


def dalitz_events_gpu(gf, spec, n, seed):
    """Accept-reject with the library's own density (normalised log P on the device)."""
    gctx, groot, gobs, th = dalitz_context(gf, spec, gf.GF_FP64, False)
    nres = len(spec["resonances"])

    def accept(s12, s13, u):
        ins = gctx.dalitz_inside(groot, s12, s13)
        out = np.zeros(len(s12), dtype=bool)
        idx = np.nonzero(ins)[0]
        if len(idx):
            gctx.set_data(groot, gobs, [s12[idx], s13[idx]])
            lp = gctx.logpdf(th)
            Gm = gctx.dalitz_gram(th, nres)
            c = np.concatenate([[1.0], th[0::2] + 1j * th[1::2]])
            N = float((c.conj() @ Gm @ c).real)
            out[idx] = u[idx] * spec["envelope"] < np.exp(lp) * N
        return out

    # candidates per batch: about what n events need (acceptance ~ 6 %), at most 2^22
    s12, s13 = synth.dalitz_events(n, accept, seed,
                                   batch=int(min(1 << 22, max(1 << 16, 24 * n))))
    gctx.close()
    return s12, s13


def dalitz_workload(gf, n, seed, precision, free_shapes, data=None):
    spec = dalitz_spec()
    s12, s13 = data if data is not None else dalitz_events_gpu(gf, spec, n, seed)
    ctx, root, obs, th = dalitz_context(gf, spec, precision, free_shapes)
    ctx.set_data(root, obs, [s12, s13])
    return ctx, root, obs, [s12, s13], th


# ---- timing ---------------------------------------------------------------------------------------
def time_steps(torch, ctx, thetas, steps, warmup, grad=True, flush=True):
    """Per-step device time (CUDA events on the context's stream), L2 flushed between steps
    with a 256 MB write; also the event-pass kernel's own time from the library."""
    st = torch.cuda.Stream()
    ctx.set_stream(st.cuda_stream)
    buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for k in range(warmup):
        (ctx.nll_grad if grad else ctx.nll)(thetas[k % len(thetas)])
    torch.cuda.synchronize()
    kern, launches, vals = [], 0, []
    # the timed region is the profiler range (ncu --profile-from-start off lists only it)
    torch.cuda.profiler.start()
    t0 = time.perf_counter()
    for k in range(steps):
        if flush:
            with torch.cuda.stream(st):
                buf.zero_()
        ev[k][0].record(st)
        r = (ctx.nll_grad if grad else ctx.nll)(thetas[k % len(thetas)])
        ev[k][1].record(st)
        vals.append(r[0] if grad else r)
        tot, sk = ctx.last_eval_times()
        kern.append(sk)
        launches += ctx.last_eval_stats()[1]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    torch.cuda.profiler.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    ctx.set_stream(0)
    return dict(step_ms=ms, kernel_ms=kern, launches=launches, wall_s=wall, values=vals)


def e2e_steps(torch, ctx, cols, thetas, steps, warmup, pipelined=True):
    """Public-API step with host buffers, pipelined for 1D data sets: step k queues the
    evaluation of its events (gf_nll_grad_start), then, while it runs, loads step k+1's
    events (gf_update_data: a swap of device buffer sets, their copy and range check done
    earlier on the library's copy stream) and queues step k+3's copy from pinned host
    memory (gf_prefetch_data, two sets ahead), then takes the NLL + gradient back to the
    host (gf_nll_grad_finish).  Events in the caller's order.  Each timed step completes
    one copy of a step's events.  Wall clock per step."""
    pinned = []
    for shift in (0, 1, 2):
        p = [torch.from_numpy(np.ascontiguousarray(np.roll(c, shift))).pin_memory() for c in cols]
        pinned.append(p)
    n = len(cols[0])

    def ptrs(k):
        return [t.data_ptr() for t in pinned[k % 3]]

    if not pipelined:  # Dalitz data sets: copy, check and evaluate in turn
        for k in range(warmup):
            ctx.update_data_ptrs(n, ptrs(k))
            ctx.nll_grad(thetas[k % len(thetas)])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            ctx.update_data_ptrs(n, ptrs(k))
            ctx.nll_grad(thetas[k % len(thetas)])
        return time.perf_counter() - t0, 8 * n * len(cols)
    ctx.update_data_ptrs(n, ptrs(0))
    ctx.prefetch_data_ptrs(n, ptrs(1))
    ctx.prefetch_data_ptrs(n, ptrs(2))
    k = 0

    def step(k):
        # the evaluation queued, the next set loaded and a later one queued while it runs
        ctx.nll_grad_start(thetas[k % len(thetas)])
        ctx.update_data_ptrs(n, ptrs(k + 1))
        ctx.prefetch_data_ptrs(n, ptrs(k + 3))
        return ctx.nll_grad_finish()

    for _ in range(warmup):
        step(k)
        k += 1
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step(k)
        k += 1
    wall = time.perf_counter() - t0
    return wall, 8 * n * len(cols)


# ---- the oracle on the host cores ------------------------------------------------------------------
def _oracle_voigt_model():
    import oracle  # CPU baseline and reference arm only
    t = synth.VOIGT_TRUTH
    m = oracle.Model1D([synth.VOIGT_RANGE])
    mu, s, w = m.param(t["mu"]), m.param(t["sigma"]), m.param(t["width"])
    x0, pw, c, f = m.param(t["x0"]), m.param(t["power"]), m.param(t["c"]), m.param(t["frac"])
    m.add([m.voigt(0, mu, s, w), m.threshold(0, x0, pw, c)], [f])
    return m


def oracle_voigt_rate(n_sample, min_seconds=10.0, max_reps=50):
    """The oracle on one core: NLL + gradient over n_sample events of the workload."""
    lo, hi = synth.VOIGT_RANGE
    x = synth.voigt_threshold_events(n_sample, **synth.VOIGT_TRUTH, lo=lo, hi=hi)
    m = _oracle_voigt_model()
    reps, t0 = 0, time.perf_counter()
    while reps < max_reps:
        m.nll([x], grad=True)
        reps += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    el = time.perf_counter() - t0
    return n_sample * reps / el, reps, el


def _oracle_worker(conn, x):
    m = _oracle_voigt_model()
    while True:
        reps = conn.recv()
        if reps is None:
            break
        t0 = time.perf_counter()
        f = 0.0
        for _ in range(reps):
            f += m.nll([x], grad=True)[0]
        conn.send((time.perf_counter() - t0, f))


class OraclePool:
    """The plain FP64 oracle over the host cores: one process per core (started with spawn,
    safe after CUDA initialisation), each holding a contiguous slice of the events; one
    step = every process evaluates NLL + gradient over its slice (the sum over slices is
    the NLL of all events)."""

    def __init__(self, x, cores=None):
        import multiprocessing as mp
        self.cores = cores or max(1, len(os.sched_getaffinity(0)))
        ctx = mp.get_context("spawn")
        self.procs, self.conns = [], []
        for sl in np.array_split(np.ascontiguousarray(x), self.cores):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_worker, args=(b, sl), daemon=True)
            pr.start()
            self.procs.append(pr)
            self.conns.append(a)

    def step(self, reps=1):
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(reps)
        f = sum(c.recv()[1] for c in self.conns)
        return time.perf_counter() - t0, f

    def close(self):
        for c in self.conns:
            c.send(None)
        for pr in self.procs:
            pr.join(timeout=10)


def cpu_baseline(unit, n_all=2_000_000, seconds=5.0):
    """The oracle as it stands, on one core and on every core of the host, on samples of
    the headline workload (events of the same distribution)."""
    rate1, reps1, el1 = oracle_voigt_rate(200_000, min_seconds=seconds)
    lo, hi = synth.VOIGT_RANGE
    x = synth.voigt_threshold_events(n_all, **synth.VOIGT_TRUTH, lo=lo, hi=hi,
                                     seed=synth.SEED_VOIGT + 77)
    pool = OraclePool(x)
    pool.step()  # workers ready
    dt, _ = pool.step()
    reps = max(1, int(seconds / max(dt, 1e-3)))
    el, _ = pool.step(reps)
    pool.close()
    rate = n_all * reps / el
    return {"value": rate, "unit": unit, "cores": pool.cores, "kind": "oracle",
            "sample": f"{reps} NLL+gradient evaluations over {n_all:,} events of the workload "
                      f"split over {pool.cores} processes ({el:.1f} s)",
            "single_core": {"value": rate1, "unit": unit, "cores": 1,
                            "sample": f"{reps1} evaluations over 200,000 events ({el1:.1f} s)"}}


def measured_fp64_tflops(torch, n=4096, reps=3):
    """cuBLAS DGEMM (torch.matmul in float64) on this GPU: context for the FP64 unit peak."""
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 1e9
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return 2.0 * n ** 3 / best / 1e12


def fp32_issue(flops_per_event, n, kern_s):
    """The implementation's FP32 flops (ncu's predicated-on FADD + FMUL + 2 x FFMA per
    event) per second against the FP32 unit peak: how busy the FP32 pipe was kept."""
    a32 = flops_per_event * n / kern_s / 1e12
    return {"flops_per_event": flops_per_event, "achieved_tflops": a32,
            "peak_tflops": FP32_PEAK_TFLOPS, "frac": a32 / FP32_PEAK_TFLOPS,
            "peak_source": "152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz"}


def voigt_roofline(torch, n, kern_s, hbm_peak, mixed=False):
    """Roofline of the headline event kernel (k_sigbkg<grad>, FP64 plan).  Headline: the
    method's work, FP64_FLOPS_PER_EVENT per event, against the FP64 unit peak (the pass
    computes FP64-accurate results on the FP32 pipe, so it can exceed the FP64 pipe's
    rate); beside it the 8 B/event against measured HBM and the implementation's FP32 flops
    (ncu) against the FP32 unit peak."""
    ach64 = FP64_FLOPS_PER_EVENT["voigt_grad"] * n / kern_s / 1e12
    hb = 8 * n / kern_s / 1e9
    rf = {"bound": "alu", "achieved": ach64, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
          "frac": ach64 / FP64_PEAK_TFLOPS,
          "traffic": TRAFFIC_PER_LAUNCH.get("voigt_grad_mixed" if mixed else "voigt_grad"),
          "kernel": ("k_sigbkg<grad, mixed plan> (FP32 per event, FP64 sums)" if mixed else
                     "k_sigbkg<grad, FP64 plan> (double-float on the FP32 pipe)"),
          "kernel_ms": kern_s * 1e3,
          "algorithmic_flops_per_event": FP64_FLOPS_PER_EVENT["voigt_grad"],
          "peak_source": "FP64 unit count: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
          "hbm": {"algorithmic_bytes_per_event": 8, "achieved_gbs": hb, "peak_gbs": hbm_peak,
                  "frac_of_measured": hb / hbm_peak}}
    try:
        rf["fp64_dgemm_measured_tflops"] = measured_fp64_tflops(torch)
    except Exception as e:  # context only
        rf["fp64_dgemm_measured_tflops"] = repr(e)[:100]
    rf["fp32_issue"] = fp32_issue(
        FP32_FLOPS_PER_EVENT["voigt_grad_mixed" if mixed else "voigt_grad"], n, kern_s)
    return rf


# ---- main -----------------------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="voigt",
                    choices=["voigt", "voigt-mixed", "exp", "dalitz", "dalitz-mixed", "dalitz-free",
                             "exp-sweep", "binned", "conv", "tddp"])
    ap.add_argument("--sweep-sizes", default="1000000,10000000,100000000,1000000000",
                    help="event counts of --workload exp-sweep")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--fits", action="store_true")
    ap.add_argument("--serve", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=5.0)
    ap.add_argument("--ref-events", type=int, default=10_000_000,
                    help="events per step of the reference arm (the oracle on the host cores)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    metric = "NLL+gradient evaluations: events x evals/s (1D composite, FP64-accurate)"
    unit = "events*evals/s"

    if args.impl == "reference":
        # The reference arm is the plain FP64 CPU oracle on every host core: the headline
        # workload's events split over one process per core, one step = NLL + gradient over
        # all of them; rank 0 only.
        if rank != 0:
            return 0
        S = args.ref_events
        lo, hi = synth.VOIGT_RANGE
        x = synth.voigt_threshold_events(S, **synth.VOIGT_TRUTH, lo=lo, hi=hi,
                                         seed=synth.SEED_VOIGT)
        pool = OraclePool(x)
        dt, _ = pool.step()  # processes started and warm
        budget = 150.0       # seconds for the timed steps: a smaller sample beyond that
        if dt * args.steps > budget and S > 100_000:
            pool.close()
            S = max(100_000, int(S * budget / (dt * args.steps)))
            x = x[:S]
            pool = OraclePool(x)
            pool.step()
        for _ in range(args.warmup):
            pool.step()
        tot = sum(pool.step()[0] for _ in range(args.steps))
        pool.close()
        value = S * args.steps / tot
        sample = (f"{S:,} events of the {10_000_000:,}-event workload per step, split over "
                  f"{pool.cores} processes (one per host core)")
        out = {"impl": "reference", "metric": metric, "value": value, "unit": unit,
               "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic",
               "config": {"workload": VOIGT_WORKLOAD, "events": 10_000_000, "free_params": 5,
                          "sample_events_per_step": S,
                          "parallelism": f"host cores x{pool.cores} (oracle)"},
               "cpu_baseline": {"value": value, "unit": unit, "cores": pool.cores,
                                "kind": "oracle", "sample": sample},
               "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return 0

    import torch
    if args.workload in ("exp-sweep", "binned", "conv", "tddp"):
        # secondary workloads alone (one JSON object: their measurements), for profiling
        torch.cuda.set_device(local)
        from paper_1311_1753_gb300 import gf
        if args.workload == "exp-sweep":
            sizes = [int(v) for v in args.sweep_sizes.split(",")]
            res = run_exp_sweep(torch, gf, sizes=sizes, steps=args.steps)
        elif args.workload == "binned":
            res = run_binned(torch, gf, steps=args.steps)
        elif args.workload == "conv":
            res = run_zach(torch, gf, steps=args.steps)
        else:
            res = run_tddp(torch, gf, steps=args.steps)
        print(json.dumps({"workload": args.workload, "result": res}))
        return 0
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1311_1753_gb300 import gf

    peaks = _peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    seed = synth.SEED_VOIGT + 1000 * rank

    # arithmetic of the timed event pass: double-float pairs of f32 (FP64-accurate: 1e-12
    # per event against the FP64 oracle, f64 in and out) for the 1D and Dalitz FP64 paths,
    # f32 amplitudes for the mixed Dalitz path
    dtype = {"dalitz-mixed": "f32", "voigt-mixed": "f32"}.get(args.workload, "df64")
    if args.workload in ("voigt", "voigt-mixed"):
        n = 10_000_000
        mixed = args.workload == "voigt-mixed"
        ctx, root, obs, cols, th0 = voigt_workload(gf, n, seed,
                                                   gf.GF_MIXED if mixed else gf.GF_FP64)
        wl = VOIGT_WORKLOAD
        if mixed:
            metric = "NLL+gradient evaluations: events x evals/s (1D composite, mixed precision)"
    elif args.workload == "exp":
        n = 100_000
        ctx, root, obs, cols, th0 = exp_workload(gf, n, synth.SEED_EXP + rank, gf.GF_FP64)
        wl = "truncated exponential, 10^5 FP64 events, analytic normalisation"
        metric = "NLL+gradient evaluations: events x evals/s (exponential, FP64-accurate)"
    else:
        # fixed-shape Dalitz (cached amplitudes, 10^6 events) or free-shape Dalitz (masses and
        # widths free: amplitudes recomputed per event, 5 x 10^6 events) in mixed precision or FP64
        mixed = args.workload == "dalitz-mixed"
        big = args.workload in ("dalitz-mixed", "dalitz-free")
        n = 5_000_000 if big else 1_000_000
        ctx, root, obs, cols, th0 = dalitz_workload(
            gf, n, synth.SEED_DALITZ_BIG if big else synth.SEED_DALITZ_EVENTS,
            gf.GF_MIXED if mixed else gf.GF_FP64, big)
        wl = ("Dalitz 8 BW resonances, 5x10^6 events, 30 free, FP32 amplitudes + FP64 sums"
              if mixed else
              "Dalitz 8 BW resonances, 5x10^6 FP64 events, 30 free (masses, widths recomputed)"
              if big else "Dalitz 8 BW resonances, 10^6 FP64 events, 16 free coefficients")
        metric = f"NLL+gradient evaluations: events x evals/s ({args.workload})"

    rng = np.random.default_rng(5)
    thetas = [th0 * (1 + 1e-4 * rng.standard_normal(len(th0))) for _ in range(8)]

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    res = time_steps(torch, ctx, thetas, args.steps, args.warmup)
    clocks = clk.stop()
    if world > 1:
        torch.distributed.barrier()
    dev_s = sum(res["step_ms"]) / 1e3
    if world > 1:
        t = torch.tensor([dev_s], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        dev_s = float(t.item())
    value = n * args.steps * world / dev_s
    kern_s = float(np.mean(res["kernel_ms"])) / 1e3

    roofline = None
    if args.workload in ("voigt", "voigt-mixed"):
        roofline = voigt_roofline(torch, n, kern_s, hbm_peak, mixed=mixed)
    elif args.workload == "dalitz":
        gbs = BYTES_PER_EVENT["dalitz_cached"] * n / kern_s / 1e9
        roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": gbs / hbm_peak, "traffic": TRAFFIC_PER_LAUNCH["dalitz_cached"],
                    "kernel": "k_dalitz_stream<DF, grad, NLL, cached-only>",
                    "kernel_ms": kern_s * 1e3,
                    "algorithmic_bytes_per_event": BYTES_PER_EVENT["dalitz_cached"],
                    "fp32_issue": fp32_issue(FP32_FLOPS_PER_EVENT["dalitz_cached"], n, kern_s)}
    elif args.workload in ("dalitz-free", "dalitz-mixed"):
        # the method's FP64 operations per event against the FP64 unit peak (FP64 plan:
        # double-float on the FP32 pipe) or, executed in FP32, the FP32 peak (mixed plan)
        ops = FP64_FLOPS_PER_EVENT["dalitz_free"] * n / kern_s / 1e12
        pk = FP32_PEAK_TFLOPS if mixed else FP64_PEAK_TFLOPS
        roofline = {"bound": "alu", "achieved": ops, "peak": pk, "unit": "TFLOP/s",
                    "frac": ops / pk,
                    "traffic": TRAFFIC_PER_LAUNCH["dalitz_mixed" if mixed else "dalitz_free"],
                    "fp32_issue": fp32_issue(FP32_FLOPS_PER_EVENT["dalitz_mixed" if mixed
                                                                  else "dalitz_free"], n, kern_s),
                    "kernel": ("k_dalitz_stream<float, grad, NLL> (FP32 amplitudes)" if mixed
                               else "k_dalitz_stream<DF, grad, NLL> (double-float pairs)"),
                    "kernel_ms": kern_s * 1e3,
                    "algorithmic_flops_per_event": FP64_FLOPS_PER_EVENT["dalitz_free"],
                    "peak_source": ("152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz" if mixed
                                    else "FP64 unit count: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz")}

    # end-to-end through the C ABI with host buffers
    e2e = None
    try:
        ksteps = max(3, args.steps // 2)
        pipe = not args.workload.startswith("dalitz")
        wall, h2d = e2e_steps(torch, ctx, cols, thetas, ksteps, 2, pipelined=pipe)
        e2e = {"value": n * ksteps / wall, "unit": unit,
               "h2d_bytes_per_step": h2d + 8 * len(th0),
               "d2h_bytes_per_step": 8 * (1 + len(th0)) + 4,
               "note": ("pipelined through the C ABI: step k's NLL + gradient queued "
                        "(gf_nll_grad_start) and taken back to the host (gf_nll_grad_finish) "
                        "while the events of steps k+1 and k+2 are copied from pinned host "
                        "memory and range-checked, one after the other, on the library's "
                        "copy stream (gf_prefetch_data, two sets ahead); step k+1's are "
                        "loaded by gf_update_data during step k's evaluation; wall clock "
                        "per step"
                        if pipe else
                        "gf_update_data from pinned host memory + gf_nll_grad in turn, wall "
                        "clock per step")}
    except Exception as e:  # report, do not hide
        e2e = {"error": repr(e)[:200]}
    ctx.close()

    extra, fit_metrics = {}, {}
    if not args.no_extra and args.workload == "voigt" and rank == 0:
        extra = run_extra(torch, gf, args)
    if (args.fits or not args.no_extra) and args.workload == "voigt" and rank == 0:
        fit_metrics["time_to_fit"] = run_fits(torch, gf, args)
    if (args.serve or not args.no_extra) and args.workload == "voigt" and rank == 0:
        fit_metrics["serving"] = run_serve(torch, gf, args)
        if args.serve:
            fit_metrics["serving_burst"] = run_serve(torch, gf, args, burst=True)

    cpu = None
    if rank == 0 and world == 1:
        cpu = cpu_baseline(unit, seconds=args.cpu_seconds)

    if rank == 0:
        out = {"metric": metric, "value": value, "unit": unit, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
               "config": {"workload": wl, "events": n, "free_params": len(th0),
                          "arithmetic": ("double-float pairs on the FP32 pipe, FP64-accurate "
                                         "(per event within 1e-12 of the FP64 oracle)"
                                         if dtype == "df64" else
                                         "FP32 per event, FP64 sums and normalisation"),
                          "l2": "flushed between steps (256 MB write)",
                          "parallelism": f"replicas x{world} (independent data sets)"},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
               "gpu_launches": res["launches"], "wall_s_timed_loop": res["wall_s"],
               "event_kernel_ms": 1e3 * kern_s}
        if extra:
            out["extra"] = extra
        if fit_metrics:
            out["fit_metrics"] = fit_metrics  # last: BASELINE's fits/s, p50/p99, mixed vs FP64
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_fits(torch, gf, args):
    """Time-to-fit (gf_fit: BFGS + fused gradient + Hessian errors) per workload.  The line
    shape (10^7 events) and the free-shape Dalitz model (5 x 10^6) in FP64 and in mixed precision (FP32 per-event arithmetic, FP64 sums, then the
    FP64 refinement) on the same data from the same start, with the mixed fit's largest
    deviation from the FP64 fit in sigma units."""
    out = {}

    def timed_fit(ctx, start, tol):
        for k, pid in enumerate(ctx.free_params()):
            ctx.set_value(pid, start[k])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = ctx.fit(tol=tol)
        torch.cuda.synchronize()
        r["seconds"] = time.perf_counter() - t0
        return r

    def pair(f, m, n):
        return {"events": n, "free_params": len(f["theta"]),
                "fp64": {"seconds": f["seconds"], "calls": f["n_calls"], "status": f["status"]},
                "mixed": {"seconds": m["seconds"], "calls": m["n_calls"], "status": m["status"],
                          "fp32_calls": m["n_calls_fast"]},
                "mixed_speedup": f["seconds"] / m["seconds"],
                "max_abs_dev_mixed_vs_fp64_in_sigma":
                    float(np.max(np.abs((m["theta"] - f["theta"]) / f["err"]))),
                "max_rel_err_diff": float(np.max(np.abs(m["err"] / f["err"] - 1)))}

    ctx, root, obs, cols, th = exp_workload(gf, 100_000, synth.SEED_EXP, gf.GF_FP64)
    r = timed_fit(ctx, np.array([-2.0]), 1e-8)
    out["exp_1e5"] = {"seconds": r["seconds"], "calls": r["n_calls"], "status": r["status"],
                              "alpha": float(r["theta"][0]), "err": float(r["err"][0])}
    ctx.close()
    res = {}
    for prec, name in ((gf.GF_FP64, "fp64"), (gf.GF_MIXED, "mixed")):
        ctx, root, obs, cols, th = voigt_workload(gf, 10_000_000, synth.SEED_VOIGT, prec)
        res[name] = timed_fit(ctx, th * np.array([1.0002, 1.1, 0.85, 1.1, 0.93]), 1e-6)
        ctx.close()
    out["voigt_1e7"] = pair(res["fp64"], res["mixed"], 10_000_000)
    out["voigt_1e7"]["pull_vs_truth_fp64"] = (
        (res["fp64"]["theta"] - th) / res["fp64"]["err"]).tolist()
    spec = dalitz_spec()
    data = dalitz_events_gpu(gf, spec, 1_000_000, synth.SEED_DALITZ_EVENTS)
    ctx, root, obs, cols, th = dalitz_workload(gf, 1_000_000, 0, gf.GF_FP64, False, data)
    rng = np.random.default_rng(8)
    r = timed_fit(ctx, th + 0.02 * rng.standard_normal(len(th)), 1e-6)
    out["dalitz_fixed_1e6"] = {"seconds": r["seconds"], "calls": r["n_calls"],
                                 "status": r["status"]}
    ctx.close()
    data5 = dalitz_events_gpu(gf, spec, 5_000_000, synth.SEED_DALITZ_BIG)
    res = {}
    for prec, name in ((gf.GF_FP64, "fp64"), (gf.GF_MIXED, "mixed")):
        ctx, root, obs, cols, th = dalitz_workload(gf, 5_000_000, 0, prec, True, data5)
        start = th * (1 + 0.01 * np.random.default_rng(9).standard_normal(len(th)))
        res[name] = timed_fit(ctx, start, 1e-8)
        ctx.close()
    out["dalitz_free_5e6"] = pair(res["fp64"], res["mixed"], 5_000_000)
    return out


def run_serve(torch, gf, args, nreq=256, burst=False):
    """Pull study through the fit server: Poisson arrivals at 20/s, event counts
    log-uniform in [1e4, 4e6], models 1D composite or Dalitz by a fair coin, each data set
    drawn at the truth from its own seed; admission by a 150 GB device budget."""
    kinds, counts, seeds = synth.serving_requests(nreq)
    arrivals = synth.poisson_arrivals(nreq, 20.0)
    spec = dalitz_spec()
    lo, hi = synth.VOIGT_RANGE
    t = synth.VOIGT_TRUTH
    reqs = []
    t_gen = time.perf_counter()
    for j in range(nreq):
        n = int(counts[j])
        if kinds[j] == 0:
            x = synth.voigt_threshold_events(n, **t, lo=lo, hi=hi, seed=int(seeds[j]))
            reqs.append(("voigt", [x]))
        else:
            s12, s13 = dalitz_events_gpu(gf, spec, n, int(seeds[j]))
            reqs.append(("dalitz", [s12, s13]))
    t_gen = time.perf_counter() - t_gen
    truth_v = np.array([t["mu"], t["sigma"], t["width"], t["c"], t["frac"]])
    srv = gf.Server(precision=gf.GF_MIXED, mem_budget=150 << 30, max_slots=64,
                    wait_timeout_s=600.0)
    tickets, truths = [], []
    t0 = time.perf_counter()
    for j, (kind, cols) in enumerate(reqs):
        while not burst and time.perf_counter() - t0 < arrivals[j]:
            time.sleep(0.0005)
        if kind == "voigt":
            ctx, root, obs, _, _ = voigt_model_nodata(gf)
            start = truth_v
        else:
            ctx, root, obs, th = dalitz_context(gf, spec, gf.GF_MIXED, False)
            start = th
        ds = ctx.make_dataset(obs, cols)
        tickets.append(srv.submit(ctx, ds, root, tol=1e-6))
        truths.append(start)
    srv.drain()
    t_all = time.perf_counter() - t0
    lat, pulls_v, pulls_d, bad = [], [], [], 0
    for j, tk in enumerate(tickets):
        r = srv.poll(tk)
        lat.append(r["latency"])
        if r["status"] != 0:
            bad += 1
            continue
        p = (r["theta"] - truths[j]) / r["err"]
        (pulls_v if kinds[j] == 0 else pulls_d).append(p)
    st = srv.stats()
    srv.close()
    lat = np.array(lat)
    pv, pd = np.array(pulls_v), np.array(pulls_d)
    return {"requests": nreq, "arrivals": "all at t=0" if burst else "Poisson 20/s",
            "fits_per_s": nreq / t_all, "wall_s": t_all,
            "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
            "not_converged": bad, "ticks": st["ticks"], "launches": st["launches"],
            "launches_per_tick": st["launches"] / max(1, st["ticks"]),
            "peak_slots": st["peak_slots"], "data_generation_s": t_gen,
            "pull_1d_mean": pv.mean(0).tolist() if len(pv) else None,
            "pull_1d_width": pv.std(0).tolist() if len(pv) else None,
            "pull_dalitz_mean_avg": float(pd.mean()) if len(pd) else None,
            "pull_dalitz_width_avg": float(pd.std(0).mean()) if len(pd) else None,
            "pull_dalitz_width_range": [float(pd.std(0).min()), float(pd.std(0).max())] if len(pd) else None,
            "precision": "mixed (FP32 per-event arithmetic, FP64 sums and normalisation) + FP64 "
                         "refinement"}


def voigt_model_nodata(gf, precision=None):
    lo, hi = synth.VOIGT_RANGE
    t = synth.VOIGT_TRUTH
    ctx = gf.Context(0, gf.GF_MIXED if precision is None else precision)
    xo = ctx.observable("dm", lo, hi)
    mu = ctx.parameter("mu", t["mu"], 1e-5, 0.143, 0.148)
    s = ctx.parameter("sigma", t["sigma"], 1e-5, 1e-5, 2e-3)
    w = ctx.parameter("width", t["width"], 1e-5, 1e-6, 1e-3)
    x0 = ctx.parameter("x0", t["x0"], 1e-4, fixed=True)
    pw = ctx.parameter("power", t["power"], 0.01, fixed=True)
    c = ctx.parameter("c", t["c"], 0.5, 0.0, 200.0)
    f = ctx.parameter("frac", t["frac"], 0.01, 0.0, 1.0)
    root = ctx.add([ctx.voigt(xo, mu, s, w), ctx.threshold(xo, x0, pw, c)], [f])
    return ctx, root, [xo], None, None


def run_exp_sweep(torch, gf, sizes=(10**6, 10**7, 10**8, 10**9), steps=20):
    """Truncated exponential at growing event counts: the event pass reads 8 B per event
    and does little arithmetic, so at large n it is bound by HBM.  The data are 10^7 draws
    at alpha = -1 tiled on the device (device columns, gf_set_data_device); NLL and
    gradient per step, L2 flushed between steps."""
    base = torch.from_numpy(synth.exp_events(10**7, -1.0, seed=synth.SEED_EXP)).cuda()
    hbm = _peaks().get("hbm_gbs", 6800.0)
    rows = []
    for n in sizes:
        reps = (n + len(base) - 1) // len(base)
        x = base.repeat(reps)[:n].contiguous() if reps > 1 else base[:n].contiguous()
        ctx = gf.Context(0, gf.GF_FP64)
        xo = ctx.observable("x", 0.0, 10.0)
        a = ctx.parameter("alpha", -1.0, 0.1, -10.0, 10.0)
        root = ctx.exp(xo, a)
        ctx.set_data_device(root, [xo], n, [x.data_ptr()], keep=x)
        r = time_steps(torch, ctx, [np.array([-1.0 - 1e-3 * k]) for k in range(4)], steps, 3)
        k_s = float(np.mean(r["kernel_ms"])) / 1e3
        rows.append({"events": n, "ms_per_eval": float(np.mean(r["step_ms"])),
                     "kernel_ms": k_s * 1e3, "kernel_gbs": 8 * n / k_s / 1e9,
                     "kernel_frac_of_measured_hbm": 8 * n / k_s / 1e9 / hbm,
                     "events_x_evals_per_s": n * steps / (sum(r["step_ms"]) / 1e3)})
        ctx.close()
        del x
    torch.cuda.empty_cache()
    return rows


def run_binned(torch, gf, nb=4000, steps=50):
    """Binned fit of the 1D composite (the paper's D*+ width fit is binned, Sec. 4): the
    10^7 events of the headline workload in 4000 bins; per metric the evaluation time
    (NLL or chi-squared + gradient) and a fit from a displaced start."""
    lo, hi = synth.VOIGT_RANGE
    t = synth.VOIGT_TRUTH
    x = synth.voigt_threshold_events(10_000_000, **t, lo=lo, hi=hi, seed=synth.SEED_VOIGT)
    counts = np.histogram(x, nb, (lo, hi))[0].astype(float)
    th0 = np.array([t["mu"], t["sigma"], t["width"], t["c"], t["frac"]])
    out = {"bins": nb, "events_binned": 10_000_000}
    for metric, name in ((gf.GF_METRIC_CHISQ, "chisq"), (gf.GF_METRIC_BINNED_NLL, "poisson")):
        ctx, root, obs, _, _ = voigt_model_nodata(gf, gf.GF_FP64)
        ctx.set_binned_data(root, obs, [nb], counts)
        ctx.set_metric(metric)
        r = time_steps(torch, ctx, [th0 * (1 + 1e-4 * k) for k in range(4)], steps, 3, flush=False)
        start = th0 * np.array([1.0002, 1.1, 0.85, 1.1, 0.93])
        for k, pid in enumerate(ctx.free_params()):
            ctx.set_value(pid, start[k])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = ctx.fit(tol=1e-6)
        sec = time.perf_counter() - t0
        out[name] = {"us_per_eval": 1e3 * float(np.mean(r["step_ms"])),
                     "kernel_us": 1e3 * float(np.mean(r["kernel_ms"])),
                     "launches_per_eval": r["launches"] / steps,
                     "fit_seconds": sec, "fit_calls": f["n_calls"], "fit_status": f["status"],
                     "pull_vs_truth": ((f["theta"] - th0) / f["err"]).tolist()}
        ctx.close()
    return out


def zach_model(gf, lattice=860, nbins=4000):
    """The paper's binned D*+ width fit (Sec. 4): a P-wave relativistic Breit-Wigner in the
    D*+ - D0 mass difference convolved with a resolution of three Gaussians, plus a
    threshold background; free: dm0, Gamma0, the three widths and two fractions of the
    resolution, the background slope and the signal fraction."""
    lo, hi = synth.VOIGT_RANGE
    ctx = gf.Context(0, gf.GF_FP64)
    x = ctx.observable("dm", lo, hi)
    r = ctx.observable("res", -0.002, 0.002)
    d0, pic = 1.86484, 0.13957
    dm0 = ctx.parameter("dm0", 0.14543, 1e-5, 0.143, 0.148)
    g0 = ctx.parameter("gamma0", 8.3e-5, 1e-5, 1e-6, 1e-3)
    cst = [ctx.parameter(nm, v, 1e-3, fixed=True)
           for nm, v in (("shift", d0), ("mD0", d0), ("mpi", pic), ("R", 1.5))]
    sig = ctx.relbw(x, dm0, g0, *cst, spin=1)
    ctx.set_norm_grid(sig, nbins)
    zero = ctx.parameter("zero", 0.0, 1e-5, fixed=True)
    s = [ctx.parameter(f"s{k}", v, 1e-5, 1e-6, 2e-3) for k, v in enumerate((2e-4, 4.5e-4, 9e-4))]
    f = [ctx.parameter("f0", 0.6, 0.01, 0.0, 1.0), ctx.parameter("f1", 0.3, 0.01, 0.0, 1.0)]
    res = ctx.add([ctx.gauss(r, zero, sk) for sk in s], f)
    conv = ctx.conv(x, sig, res, lattice)
    x0 = ctx.parameter("x0", lo, 1e-4, fixed=True)
    pw = ctx.parameter("power", 0.5, 0.01, fixed=True)
    c = ctx.parameter("c", 20.0, 0.5, 0.0, 200.0)
    fs = ctx.parameter("fsig", 0.3, 0.01, 0.0, 1.0)
    th = ctx.threshold(x, x0, pw, c)
    ctx.set_norm_grid(th, nbins)
    root = ctx.add([conv, th], [fs])
    return ctx, root, [x]


def run_zach(torch, gf, nb=4000, steps=50):
    """Binned chi-squared fit of the line shape x resolution + background on the 10^7
    events of the headline workload in 4000 bins: evaluation time (norm grids, the two
    convolution launches, the bin pass) and a fit from a displaced start."""
    lo, hi = synth.VOIGT_RANGE
    x = synth.voigt_threshold_events(10_000_000, **synth.VOIGT_TRUTH, lo=lo, hi=hi,
                                     seed=synth.SEED_VOIGT)
    counts = np.histogram(x, nb, (lo, hi))[0].astype(float)
    ctx, root, obs = zach_model(gf)
    ctx.set_binned_data(root, obs, [nb], counts)
    ctx.set_metric(gf.GF_METRIC_CHISQ)
    th0 = np.array([ctx.value(p) for p in ctx.free_params()])
    r = time_steps(torch, ctx, [th0 * (1 + 1e-4 * k) for k in range(4)], steps, 3, flush=False)
    start = th0 * np.array([1.0001, 1.2, 1.1, 0.9, 1.05, 0.95, 1.02, 1.1, 0.9])
    for k, pid in enumerate(ctx.free_params()):
        ctx.set_value(pid, start[k])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f = ctx.fit(tol=1e-6)
    sec = time.perf_counter() - t0
    out = {"bins": nb, "lattice": 860, "resolution_offsets": 161, "free_params": len(th0),
           "us_per_eval": 1e3 * float(np.mean(r["step_ms"])),
           "event_kernel_us": 1e3 * float(np.mean(r["kernel_ms"])),
           "launches_per_eval": r["launches"] / steps,
           "fit_seconds": sec, "fit_calls": f["n_calls"], "fit_status": f["status"],
           "chi2_per_bin": f["nll"] / nb}
    ctx.close()
    return out


def run_tddp(torch, gf, n=100_000, steps=30):
    """The paper's driver, the time-dependent Dalitz (mixing) fit of D0 -> pi+ pi- pi0
    (Sec. 4: ~10^5 events): the 8-resonance model for D0 and D0bar, decay time with tau,
    x, y and a per-event resolution sigma_t (uniform in [0.05, 0.15] ps) scaled by s;
    20 free parameters (16 coefficients, tau, x, y, s), 256 x 256 normalisation grid.
    Events: (s12, s13) drawn with the library's Dalitz density, t = exponential(tau) +
    Gaussian(sigma_t).  Evaluation time (NLL + gradient) and a fit from a displaced start."""
    spec = dalitz_spec()
    s12, s13 = dalitz_events_gpu(gf, spec, n, synth.SEED_DALITZ_EVENTS + 7)
    rng = np.random.Generator(np.random.PCG64(synth.SEED_DALITZ_EVENTS + 8))
    sigt = rng.uniform(0.05, 0.15, n)
    t = np.clip(rng.exponential(0.41, n) + sigt * rng.standard_normal(n), -1.9, 19.0)
    ctx = gf.Context(0, gf.GF_FP64)
    o12 = ctx.observable("s12", 0.0, 4.0)
    o13 = ctx.observable("s13", 0.0, 4.0)
    ot = ctx.observable("t", -2.0, 20.0)
    osg = ctx.observable("sigt", 0.0, 1.0)
    res = []
    for i, r in enumerate(spec["resonances"]):
        m0 = ctx.parameter(f"m0_{i}", r["m0"], 0.005, fixed=True)
        g0 = ctx.parameter(f"g0_{i}", r["g0"], 0.005, fixed=True)
        re = ctx.parameter(f"re_{i}", r["re"], 0.01)
        im = ctx.parameter(f"im_{i}", r["im"], 0.01)
        res.append(dict(channel=r["channel"], spin=r["spin"], mass=m0, width=g0, re=re, im=im))
    tau = ctx.parameter("tau", 0.41, 0.01, 0.05, 5.0)
    mx = ctx.parameter("x", 0.0, 0.01, -1.0, 1.0)
    my = ctx.parameter("y", 0.0, 0.01, -1.0, 1.0)
    sc = ctx.parameter("scale", 1.0, 0.01, 0.1, 5.0)
    root = ctx.tddp(o12, o13, ot, osg, spec["kin"], res, tau, mx, my, sc)
    ctx.set_data(root, [o12, o13, ot, osg], [s12, s13, t, sigt])
    th0 = np.array([ctx.value(p) for p in ctx.free_params()])
    r = time_steps(torch, ctx, [th0 + 1e-4 * k for k in range(4)], steps, 3)
    start = th0 + 0.02 * np.random.default_rng(3).standard_normal(len(th0))
    for k, pid in enumerate(ctx.free_params()):
        ctx.set_value(pid, start[k])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f = ctx.fit(tol=1e-6)
    sec = time.perf_counter() - t0
    fp = ctx.free_params()
    out = {"events": n, "free_params": len(th0), "grid": "256 x 256",
           "ms_per_eval": float(np.mean(r["step_ms"])),
           "event_kernel_ms": float(np.mean(r["kernel_ms"])),
           "events_x_evals_per_s": n * steps / (sum(r["step_ms"]) / 1e3),
           "fit_seconds": sec, "fit_calls": f["n_calls"], "fit_status": f["status"],
           "tau_x_y_scale": f["theta"][-4:].tolist(), "errors": f["err"][-4:].tolist()}
    ctx.close()
    return out


def run_extra(torch, gf, args):
    """Secondary measurements: exponential, binned, mixing and Dalitz evaluation rates (and, on request, fit
    times and the serving study)."""
    out = {}
    K = max(5, args.steps)
    # truncated exponential, 10^5 events
    ctx, root, obs, cols, th = exp_workload(gf, 100_000, synth.SEED_EXP, gf.GF_FP64)
    r = time_steps(torch, ctx, [th * (1 + 1e-3 * k) for k in range(4)], 50, 5, flush=False)
    out["exp_1e5"] = {"events_x_evals_per_s": 1e5 * 50 / (sum(r["step_ms"]) / 1e3),
                              "us_per_eval": 1e3 * float(np.mean(r["step_ms"])),
                              "kernel_us": 1e3 * float(np.mean(r["kernel_ms"]))}
    ctx.close()
    out["exp_hbm_sweep"] = run_exp_sweep(torch, gf)
    out["binned_voigt_4000"] = run_binned(torch, gf)
    out["binned_relbw_conv_4000"] = run_zach(torch, gf)
    out["tddp_mixing_1e5"] = run_tddp(torch, gf)
    # fixed-shape Dalitz (FP64, 1e6 events, cached per-event amplitudes, Gram normalisation)
    spec = dalitz_spec()
    data = dalitz_events_gpu(gf, spec, 1_000_000, synth.SEED_DALITZ_EVENTS)
    ctx, root, obs, cols, th = dalitz_workload(gf, 1_000_000, 0, gf.GF_FP64, False, data)
    rng = np.random.default_rng(2)
    ths = [th * (1 + 1e-3 * rng.standard_normal(len(th))) for _ in range(4)]
    r = time_steps(torch, ctx, ths, K, 3)
    out["dalitz_fixed_fp64_1e6"] = {
        "events_x_evals_per_s": 1e6 * K / (sum(r["step_ms"]) / 1e3),
        "ms_per_eval": float(np.mean(r["step_ms"])), "kernel_ms": float(np.mean(r["kernel_ms"]))}
    ctx.close()
    # free-shape Dalitz data: 5e6 events; mixed vs FP64 on the same data, 30 free parameters
    data5 = dalitz_events_gpu(gf, spec, 5_000_000, synth.SEED_DALITZ_BIG)
    for prec, name in ((gf.GF_MIXED, "mixed"), (gf.GF_FP64, "fp64")):
        ctx, root, obs, cols, th = dalitz_workload(gf, 5_000_000, 0, prec, True, data5)
        ths = [th * (1 + 1e-3 * rng.standard_normal(len(th))) for _ in range(4)]
        r = time_steps(torch, ctx, ths, K, 3)
        out[f"dalitz_free_{name}_5e6"] = {
            "events_x_evals_per_s": 5e6 * K / (sum(r["step_ms"]) / 1e3),
            "ms_per_eval": float(np.mean(r["step_ms"])),
            "kernel_ms": float(np.mean(r["kernel_ms"])), "free_params": len(th)}
        ctx.close()
    m, f = out["dalitz_free_mixed_5e6"], out["dalitz_free_fp64_5e6"]
    out["dalitz_free_mixed_over_fp64_speedup"] = f["ms_per_eval"] / m["ms_per_eval"]
    return out


if __name__ == "__main__":
    sys.exit(main())
