"""The fit server: every request's result is the same alone (gf_fit) and in the mix
(FP64: bitwise; mixed precision: within 1e-9 relative), admission respects the slot cap
and the memory budget, and results arrive for requests submitted while others run."""
from __future__ import annotations

import time

import numpy as np
import pytest

from paper_1311_1753_gb300 import synth
from tests import oracle_models as om
from tests import product_models as pm

pytestmark = pytest.mark.gpu
SPEC = om.load_dalitz_spec()


@pytest.fixture(scope="module")
def gf():
    from paper_1311_1753_gb300 import gf as _gf
    return _gf


def _requests(gf, precision, k=6):
    lo, hi = synth.VOIGT_RANGE
    d_full = om.dalitz_from_spec(SPEC)
    reqs = []
    for j in range(k):
        if j % 2 == 0:
            n = [20_000, 60_000, 35_000][j // 2 % 3]
            x = synth.voigt_threshold_events(n, **synth.VOIGT_TRUTH, lo=lo, hi=hi, seed=1_000_000 + j)
            reqs.append(("voigt", [x], dict(nbins=2000)))
        else:
            n = [3000, 8000, 5000][j // 2 % 3]
            s = synth.dalitz_events(n, om.dalitz_accept(d_full, SPEC["envelope"]), seed=1_000_000 + j)
            reqs.append(("dalitz", list(s), dict(nbx=96, nby=96)))
    return reqs


def _build(gf, kind, precision, opts):
    if kind == "voigt":
        ctx, root, obs = pm.voigt_model(gf, precision=precision, nbins=opts["nbins"])
        start = np.array([0.14551, 3.2e-4, 7e-5, 21.0, 0.29])
    else:
        ctx, root, obs = pm.dalitz_model(gf, SPEC, precision=precision, nbx=opts["nbx"],
                                         nby=opts["nby"])
        th = np.array([v for r in SPEC["resonances"] for v in (r["re"], r["im"])])
        start = th + 0.01
    for k, pid in enumerate(ctx.free_params()):
        ctx.set_value(pid, start[k])
    return ctx, root, obs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_server_alone_equals_mix(gf, precision):
    prec = gf.GF_FP64 if precision == "fp64" else gf.GF_MIXED
    reqs = _requests(gf, prec)
    # EDM tolerance: 1e-8 in FP64; MINUIT-like 1e-5 when the likelihood carries FP32 noise
    tol = 1e-8 if prec == gf.GF_FP64 else 1e-5
    alone = []
    for kind, cols, opts in reqs:
        ctx, root, obs = _build(gf, kind, prec, opts)
        ctx.set_data(root, obs, cols)
        alone.append(ctx.fit(tol=tol))
        ctx.close()
    srv = gf.Server(precision=prec, mem_budget=8 << 30, max_slots=4)
    tickets = []
    for i, (kind, cols, opts) in enumerate(reqs):
        ctx, root, obs = _build(gf, kind, prec, opts)
        ds = ctx.make_dataset(obs, cols)
        tickets.append(srv.submit(ctx, ds, root, tol=tol))
        if i == 2:
            time.sleep(0.05)  # later requests arrive while the first ones run
    srv.drain()
    st = srv.stats()
    assert 1 <= st["peak_slots"] <= 4 and st["ticks"] > 0
    # every 1D evaluation and a Dalitz fit's after its first join the batched tick: at
    # most four persistent launches here (1D normalisation, signal + background events in
    # the server's precision and in FP64 for refinement steps, Dalitz events) per tick
    assert st["launches"] <= 4 * st["ticks"] + 2 * len(reqs) * 4, st
    for a, t in zip(alone, tickets):
        r = srv.poll(t)
        assert r is not None and r["status"] == gf.GF_OK
        if prec == gf.GF_FP64:
            assert np.array_equal(r["theta"], a["theta"]) and r["nll"] == a["nll"]
        else:
            assert np.allclose(r["theta"], a["theta"], rtol=1e-9, atol=0)
        assert r["latency"] > 0
    srv.close()


def test_server_memory_budget_limits_slots(gf):
    reqs = _requests(gf, gf.GF_MIXED, k=4)
    # each request needs > 5 MB (4 MB of work buffers, a Voigtian fit also its 2.6 MB table
    # of w expansions) and at most 8.5 MB: a 10 MB budget admits one at a time
    srv = gf.Server(precision=gf.GF_MIXED, mem_budget=10 << 20, max_slots=8)
    tickets = []
    for kind, cols, opts in reqs:
        ctx, root, obs = _build(gf, kind, gf.GF_MIXED, opts)
        ds = ctx.make_dataset(obs, cols)
        tickets.append(srv.submit(ctx, ds, root, tol=1e-6))
    srv.drain()
    assert srv.stats()["peak_slots"] == 1
    assert all(srv.poll(t)["status"] == gf.GF_OK for t in tickets)
    srv.close()


def _tree_model(gf, kind):
    """1D trees outside the signal + background form: an AddPdf of three leaves (the
    AddPdf-of-leaves event path) and a nested sum (the stack machine)."""
    ctx = gf.Context()
    x = ctx.observable("x", -1.0, 2.0)
    names = ["mu", "s", "ax", "a0", "a1", "f1", "f2"]
    vals = [0.4, 0.3, -0.7, 1.0, 0.3, 0.5, 0.2]
    P = [ctx.parameter(nm, v, 0.01, *((0.0, 1.0) if nm[0] == "f" else (0.0, 0.0)))
         for nm, v in zip(names, vals)]
    g, e, q = ctx.gauss(x, P[0], P[1]), ctx.exp(x, P[2]), ctx.poly(x, [P[3], P[4]])
    ctx.set_fixed(P[3], True)
    if kind == "mix3":
        root = ctx.add([g, e, q], [P[5], P[6]])
    else:
        root = ctx.add([g, ctx.add([e, q], [P[6]])], [P[5]])
    return ctx, root, [x]


def test_server_1d_tree_kinds_alone_equals_mix(gf):
    """Fits of the two general 1D event paths (their own tick kernels) beside each other
    and beside signal + background fits: FP64 results are the same bits alone and in the
    mix, and every evaluation, the first included, runs in the batched tick."""
    rng = np.random.default_rng(31)
    jobs = []
    for j in range(6):
        n = 40_000 + 10_000 * j
        x = np.where(rng.random(n) < 0.5, rng.normal(0.4, 0.3, n), rng.uniform(-1.0, 2.0, n))
        x = np.clip(x, -0.999, 1.999)
        jobs.append((["mix3", "nested"][j % 2], x))
    lo, hi = synth.VOIGT_RANGE
    jobs.append(("voigt", synth.voigt_threshold_events(30_000, **synth.VOIGT_TRUTH, lo=lo, hi=hi,
                                                       seed=77)))

    def build(kind):
        if kind == "voigt":
            ctx, root, obs = pm.voigt_model(gf, nbins=2000)
            for k, pid in enumerate(ctx.free_params()):
                ctx.set_value(pid, [0.14551, 3.2e-4, 7e-5, 21.0, 0.29][k])
            return ctx, root, obs
        return _tree_model(gf, kind)

    alone = []
    for kind, x in jobs:
        ctx, root, obs = build(kind)
        ctx.set_data(root, obs, [x])
        alone.append(ctx.fit(tol=1e-8))
        ctx.close()
    srv = gf.Server(precision=gf.GF_FP64, mem_budget=8 << 30, max_slots=8)
    tickets = []
    for kind, x in jobs:
        ctx, root, obs = build(kind)
        tickets.append(srv.submit(ctx, ctx.make_dataset(obs, [x]), root, tol=1e-8))
    srv.drain()
    st = srv.stats()
    # per tick at most: 1D normalisation, stack machine, AddPdf of leaves, signal + background
    assert st["launches"] <= 4 * st["ticks"], st
    for a, t in zip(alone, tickets):
        r = srv.poll(t)
        assert r["status"] == a["status"]
        assert np.array_equal(r["theta"], a["theta"]) and r["nll"] == a["nll"]
    srv.close()
