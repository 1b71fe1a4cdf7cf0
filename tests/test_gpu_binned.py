"""Binned fits on the sm_103a path (Sec. 2: the metric is applied to the PDF's value at
each point, so one PDF serves maximum-likelihood and chi-squared fits; Sec. 4: the binned
D*+ line-width fit) against the FP64 oracle.

Tolerances: 1e-9 relative on the metric, gradients 1e-9 of their scale (as for the
unbinned NLL); fitted parameters within 0.01 sigma of the oracle's fit."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import minimise
from paper_1311_1753_gb300 import synth
from tests import oracle_models as om
from tests import product_models as pm

pytestmark = pytest.mark.gpu
LO, HI = synth.VOIGT_RANGE


@pytest.fixture(scope="module")
def gf():
    from paper_1311_1753_gb300 import gf as _gf
    return _gf


def _hist(nb, n=400_000, seed=11):
    x = synth.voigt_threshold_events(n, **synth.VOIGT_TRUTH, lo=LO, hi=HI, seed=seed)
    counts, edges = np.histogram(x, nb, (LO, HI))
    return 0.5 * (edges[1:] + edges[:-1]), counts.astype(float)


def _close(a, b, rel=1e-9):
    assert abs(a - b) <= rel * max(1.0, abs(b)), (a, b)


def _grad_close(g, go, rel=1e-9):
    scale = np.abs(go).max()
    assert np.all(np.abs(g - go) <= rel * np.maximum(np.abs(go), 1e-3 * scale) + 1e-12 * scale), (g, go)


@pytest.mark.parametrize("nb", [1, 7, 1000, 4096])
@pytest.mark.parametrize("metric", [0, 1, 2])
def test_binned_voigt_metrics_parity(gf, nb, metric):
    c, n = _hist(nb)
    ctx, root, obs = pm.voigt_model(gf, nbins=2000)
    ctx.set_binned_data(root, obs, [nb], n)
    ctx.set_metric(metric)
    m, free = om.voigt_model(nbins=2000)
    K = n.sum() * (HI - LO) / nb
    for scale in (np.array([1.0, 1.0, 1.0, 1.0, 1.0]), np.array([1.00002, 1.03, 0.96, 1.05, 0.95])):
        th = m.p[free] * scale
        p = m.p.copy(); p[free] = th
        f, g = ctx.nll_grad(th)
        fo, go = m.binned([c], n, K, metric, s2=np.maximum(n, 1.0), p=p, grad=True)
        _close(f, fo)
        _close(ctx.nll(th), f, 1e-12)
        # one bin: its centre lies 16 sigma into the Voigtian's tail, where d V/d sigma is
        # a difference of terms ~3e5 times larger (the Lorentzian tail barely depends on
        # sigma); pair arithmetic (~1e-14) then leaves ~3e-9 of it
        _grad_close(g, go[free], rel=1e-8 if nb == 1 else 1e-9)


@pytest.mark.parametrize("metric", [0, 1, 2])
def test_binned_2d_log_domain_and_errors(gf, metric):
    """ProdPdf over two binned observables (log-domain root), user-given errors."""
    rng = np.random.default_rng(5)
    nbx, nby = 40, 30
    counts = rng.poisson(50.0 * np.outer(np.exp(-0.3 * np.arange(nbx) / 4), np.ones(nby))).astype(float)
    errors = np.sqrt(counts + 2.0)
    ctx = gf.Context()
    x = ctx.observable("x", 0.0, 10.0)
    y = ctx.observable("y", -2.0, 3.0)
    a = ctx.parameter("a", -0.3, 0.1, -10, 10)
    mu = ctx.parameter("mu", 0.4, 0.1)
    s = ctx.parameter("s", 1.9, 0.1, 0.01, 9)
    root = ctx.prod([ctx.exp(x, a), ctx.gauss(y, mu, s)])
    ctx.set_binned_data(root, [x, y], [nbx, nby], counts, errors)
    ctx.set_metric(metric)
    m = oracle.Model1D([(0.0, 10.0), (-2.0, 3.0)])
    m.prod([m.exp(0, m.param(-0.3)), m.gauss(1, m.param(0.4), m.param(1.9))])
    cx = (np.arange(nbx) + 0.5) * 10.0 / nbx
    cy = -2.0 + (np.arange(nby) + 0.5) * 5.0 / nby
    X, Y = np.meshgrid(cx, cy, indexing="ij")
    K = counts.sum() * (10.0 / nbx) * (5.0 / nby)
    th = np.array([-0.31, 0.35, 2.1])
    f, g = ctx.nll_grad(th)
    fo, go = m.binned([X.ravel(), Y.ravel()], counts.ravel(), K, metric, s2=errors.ravel() ** 2,
                      p=th, grad=True)
    _close(f, fo)
    _grad_close(g, go)


def test_binned_zero_density_bins(gf):
    """Bins below the threshold's x0 have P = 0 (and no entries): finite metrics, and the
    chi-squared gradient there still counts (its factor does not divide by P)."""
    t = dict(synth.VOIGT_TRUTH)
    t["x0"] = LO + 0.004
    x = synth.voigt_threshold_events(200_000, **t, lo=LO, hi=HI, seed=3)
    counts, edges = np.histogram(x, 500, (LO, HI))
    c = 0.5 * (edges[1:] + edges[:-1])
    n = counts.astype(float)
    n[c < t["x0"]] = 0.0
    # a threshold-only model: P = 0 below x0
    ctx = gf.Context()
    xo = ctx.observable("dm", LO, HI)
    x0 = ctx.parameter("x0", t["x0"], 1e-4, fixed=True)
    pw = ctx.parameter("power", 0.5, 0.01, fixed=True)
    cc = ctx.parameter("c", 20.0, 0.5, 0.0, 200.0)
    root = ctx.threshold(xo, x0, pw, cc)
    ctx.set_norm_grid(root, 2000)
    ctx.set_binned_data(root, [xo], [500], n)
    m = oracle.Model1D([(LO, HI)], nbins=2000)
    m.threshold(0, m.param(t["x0"]), m.param(0.5), m.param(20.0))
    K = n.sum() * (HI - LO) / 500
    for metric in (0, 1, 2):
        ctx.set_metric(metric)
        f, g = ctx.nll_grad(np.array([22.0]))
        p = m.p.copy(); p[2] = 22.0
        fo, go = m.binned([c], n, K, metric, s2=np.maximum(n, 1.0), p=p, grad=True)
        assert np.isfinite(f)
        _close(f, fo)
        _grad_close(g, go[[2]])


def test_binned_chisq_fit_matches_oracle_fit(gf):
    """A chi-squared fit of the 1D composite histogram (4000 bins, the size of the
    paper's binned fit) by gf_fit lands within 0.01 sigma of the oracle's BFGS fit, with
    errors from Delta chi2 = 1 within 1 %."""
    nb = 4000
    c, n = _hist(nb, n=2_000_000, seed=21)
    ctx, root, obs = pm.voigt_model(gf, nbins=4000)
    ctx.set_binned_data(root, obs, [nb], n)
    ctx.set_metric(gf.GF_METRIC_CHISQ)
    m, free = om.voigt_model(nbins=4000)
    start = m.p[free] * np.array([1.0001, 1.05, 0.9, 1.05, 0.95])
    for k, pid in enumerate(ctx.free_params()):
        ctx.set_value(pid, start[k])
    r = ctx.fit(tol=1e-10)
    assert r["status"] == gf.GF_OK
    K = n.sum() * (HI - LO) / nb
    s2 = np.maximum(n, 1.0)

    def fg(q):
        p = m.p.copy(); p[free] = q
        f, g = m.binned([c], n, K, 2, s2=s2, p=p, grad=True)
        return f, g[free]
    lo = np.array([0.143, 1e-5, 1e-6, 0.0, 0.0])
    hi = np.array([0.148, 2e-3, 1e-3, 200.0, 1.0])
    step = np.array([1e-5, 1e-5, 1e-5, 0.5, 0.01])
    ro = minimise.fit(fg, start, step, lo, hi, up=1.0, tol=1e-10)
    assert ro.converged
    assert np.all(np.abs(r["theta"] - ro.x) <= 0.01 * ro.err), (r["theta"], ro.x, ro.err)
    assert np.all(np.abs(r["err"] / ro.err - 1) < 0.01)


def test_binned_rejections(gf):
    ctx, root, obs = pm.voigt_model(gf, nbins=2000)
    with pytest.raises(gf.GFError):
        ctx.make_binned_dataset(obs, [10], -np.ones(10))
    with pytest.raises(gf.GFError):
        ctx.make_binned_dataset(obs, [10], np.ones(10), errors=np.zeros(10))
    x = synth.voigt_threshold_events(1000, **synth.VOIGT_TRUTH, lo=LO, hi=HI)
    ctx.set_data(root, obs, [x])
    ctx.set_metric(gf.GF_METRIC_CHISQ)  # unbinned data: refused at the evaluation
    th = np.array([0.1455, 3e-4, 8e-5, 20.0, 0.3])
    with pytest.raises(gf.GFError):
        ctx.nll(th)
    ctx.set_metric(gf.GF_METRIC_NLL)
    assert np.isfinite(ctx.nll(th))
    c, n = _hist(100)
    ctx.set_binned_data(root, obs, [100], n)
    with pytest.raises(gf.GFError):
        ctx.update_data([c])


def test_binned_fits_in_the_server_equal_alone(gf):
    """Binned chi-squared and Poisson fits join the batched tick beside unbinned ones:
    FP64 results are the same bits alone and in the mix."""
    jobs = []
    for j in range(4):
        c, n = _hist(1500 + 500 * j, n=300_000, seed=100 + j)
        jobs.append(("binned", n, [gf.GF_METRIC_CHISQ, gf.GF_METRIC_BINNED_NLL][j % 2]))
        x = synth.voigt_threshold_events(30_000, **synth.VOIGT_TRUTH, lo=LO, hi=HI, seed=200 + j)
        jobs.append(("unbinned", x, gf.GF_METRIC_NLL))
    start = np.array([0.14551, 3.2e-4, 7e-5, 21.0, 0.29])

    def build(kind, data, metric):
        ctx, root, obs = pm.voigt_model(gf, nbins=2000)
        for k, pid in enumerate(ctx.free_params()):
            ctx.set_value(pid, start[k])
        ctx.set_metric(metric)
        return ctx, root, obs

    alone = []
    for kind, data, metric in jobs:
        ctx, root, obs = build(kind, data, metric)
        if kind == "binned":
            ctx.set_binned_data(root, obs, [len(data)], data)
        else:
            ctx.set_data(root, obs, [data])
        alone.append(ctx.fit(tol=1e-8))
        ctx.close()
    srv = gf.Server(precision=gf.GF_FP64, mem_budget=4 << 30, max_slots=8)
    tickets = []
    for kind, data, metric in jobs:
        ctx, root, obs = build(kind, data, metric)
        ds = (ctx.make_binned_dataset(obs, [len(data)], data) if kind == "binned"
              else ctx.make_dataset(obs, [data]))
        tickets.append(srv.submit(ctx, ds, root, tol=1e-8))
    srv.drain()
    for a, t in zip(alone, tickets):
        r = srv.poll(t)
        assert r["status"] == gf.GF_OK and a["status"] == gf.GF_OK
        assert np.array_equal(r["theta"], a["theta"]) and r["nll"] == a["nll"]
    srv.close()
