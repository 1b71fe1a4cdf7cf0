"""Parity of the sm_103a 1D path with the FP64 oracle (truncated exponential, Voigtian + threshold, generic trees).

Tolerances: 1e-12 relative per event on P (|log P_gpu - log P_orc| <= 1e-12 for every
event), 1e-9 relative on the total NLL, gradients 1e-9 relative to the gradient's scale."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1311_1753_gb300 import synth
from tests import oracle_models as om
from tests import product_models as pm
from tests.parity import per_event

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    from paper_1311_1753_gb300 import gf as _gf
    return _gf


def _theta(values, free):
    return np.array([values[i] for i in free], dtype=float)


def _grad_close(g_gpu, g_orc, n, rel=1e-9):
    scale = np.maximum(np.abs(g_orc), 1e-6 * n)
    assert np.all(np.abs(g_gpu - g_orc) <= rel * scale + 1e-9 * np.abs(g_orc).max()), (g_gpu, g_orc)


# ---- truncated exponential ------------------------------------------------------------------------
@pytest.mark.parametrize("n", [0, 1, 2, 31, 33, 257, 100_000, 1_000_003])
def test_exponential_parity(gf, n):
    x = synth.exp_events(max(n, 1), -1.0)[:n]
    ctx, root, obs = pm.exp_model(gf, -2.0)
    ctx.set_data(root, obs, [x])
    m, free = om.exp_model(-2.0)
    for alpha in (-1.0, -2.0, 0.3, 1e-6, -9.5):
        th = np.array([alpha])
        p = m.p.copy(); p[free] = th
        lg = ctx.logpdf(th)
        if n:
            lo = m.logpdf([x], p)
            per_event(f"exponential n={n} alpha={alpha}", lg, lo)
        f, g = ctx.nll_grad(th)
        fo, go = m.nll([x], p, grad=True)
        assert abs(f - fo) <= 1e-9 * max(1.0, abs(fo))
        assert abs(ctx.nll(th) - f) <= 1e-12 * max(1.0, abs(f))
        if n:
            assert abs(g[0] - go[0]) <= 1e-9 * max(abs(go[0]), n * 1e-6)


def test_exponential_deterministic_bitwise(gf):
    x = synth.exp_events(100_000, -1.0)
    ctx, root, obs = pm.exp_model(gf)
    ctx.set_data(root, obs, [x])
    vals = {ctx.nll(np.array([-1.1])) for _ in range(5)}
    assert len(vals) == 1


# ---- Voigtian + threshold --------------------------------------------------------------------
def _voigt_data(n, seed=synth.SEED_VOIGT):
    lo, hi = synth.VOIGT_RANGE
    return synth.voigt_threshold_events(n, **synth.VOIGT_TRUTH, lo=lo, hi=hi, seed=seed)


@pytest.mark.parametrize("n", [1, 33, 4099, 200_000])
def test_voigt_parity(gf, n):
    x = _voigt_data(n)
    ctx, root, obs = pm.voigt_model(gf)
    ctx.set_data(root, obs, [x])
    m, free = om.voigt_model()
    base = m.p.copy()
    for scale in ([1, 1, 1, 1, 1], [1.00002, 1.05, 0.9, 1.1, 0.95]):
        p = base.copy()
        p[free] = base[free] * np.array(scale)
        th = p[free]
        lo_ = m.logpdf([x], p)
        lg = ctx.logpdf(th)
        per_event(f"voigt n={n}", lg, lo_)
        f, g = ctx.nll_grad(th)
        fo, go = m.nll([x], p, grad=True)
        assert abs(f - fo) <= 1e-9 * abs(fo)
        _grad_close(g, go[free], n)


def test_voigt_free_shape_parameters(gf):
    # x0 and power free as well (fixed in the workload, free in general)
    x = _voigt_data(20_000)
    ctx, root, obs = pm.voigt_model(gf, free_shape=True, nbins=2000)
    ctx.set_data(root, obs, [x])
    m, _ = om.voigt_model(nbins=2000)
    p = m.p.copy()
    p[3] = synth.VOIGT_RANGE[0] - 2e-4
    p[4] = 0.6
    th = p.copy()  # every parameter is free here, in creation order
    f, g = ctx.nll_grad(th)
    fo, go = m.nll([x], p, grad=True)
    assert abs(f - fo) <= 1e-9 * abs(fo)
    _grad_close(g, go, len(x), rel=1e-8)


def test_voigt_full_size(gf):
    """10^7 events in the benchmark's launch shape (sorted layout, chunked w): total NLL
    against the oracle's full sum, and log P of every event against the oracle's."""
    x = _voigt_data(10_000_000)
    ctx, root, obs = pm.voigt_model(gf)
    ctx.set_data(root, obs, [x])
    m, free = om.voigt_model()
    th = m.p[free]
    f = ctx.nll(th)
    fo = m.nll([x], m.p)
    assert abs(f - fo) <= 1e-9 * abs(fo)
    per_event("voigt full 1e7", ctx.logpdf(th), m.logpdf([x], m.p))


def test_sorted_layout_matches_strided_loop(gf):
    """Events sorted by the Voigtian's observable (chunked loop, w expanded once per chunk
    of 24 events) and events in the caller's order (strided loop, w per event): the same
    NLL, gradient and per-event log P (returned in the caller's order); new events from
    gf_update_data are taken in their order, then sorted again on the second evaluation."""
    x = _voigt_data(2_000_003)
    a, ra, oa = pm.voigt_model(gf, nbins=2000)
    a.set_data(ra, oa, [x])
    b, rb, ob = pm.voigt_model(gf, nbins=2000)
    b.set_event_sort(False)
    b.set_data(rb, ob, [x])
    t = synth.VOIGT_TRUTH
    th0 = np.array([t["mu"], t["sigma"], t["width"], t["c"], t["frac"]])
    for k in range(3):
        th = th0 * np.array([1.0, 1.0 + 0.05 * k, 1.0 - 0.1 * k, 1.0, 1.0])
        fa, ga = a.nll_grad(th)
        fb, gb = b.nll_grad(th)
        assert abs(fa - fb) <= 1e-12 * abs(fb)
        _grad_close(ga, gb, len(x), rel=1e-10)
        assert abs(a.nll(th) - fb) <= 1e-12 * abs(fb)
        la, lb = a.logpdf(th), b.logpdf(th)
        per_event("sorted vs strided", la, lb, tol=2e-12)
    y = _voigt_data(2_000_003, seed=synth.SEED_VOIGT + 100)
    a.update_data([y])
    b.update_data([y])
    for _ in range(3):  # caller order, then sorted again from the second evaluation
        fa, ga = a.nll_grad(th0)
        fb, gb = b.nll_grad(th0)
        assert abs(fa - fb) <= 1e-12 * abs(fb)
        _grad_close(ga, gb, len(y), rel=1e-10)
    la, lb = a.logpdf(th0), b.logpdf(th0)
    per_event("sorted vs strided, updated data", la, lb, tol=2e-12)


def _mix3_models(gf):
    """AddPdf of three leaves, two of them in the log domain: f1 Gauss + f2 Exp + rest Poly."""
    ctx = gf.Context()
    m = oracle.Model1D([(-1.0, 2.0)])
    x = ctx.observable("x", -1.0, 2.0)
    vals = [0.4, 0.3, -0.7, 1.0, 0.3, 0.5, 0.2]
    names = ["mu", "s", "ax", "a0", "a1", "f1", "f2"]
    P = [ctx.parameter(nm, v, 0.01) for nm, v in zip(names, vals)]
    O = [m.param(v) for v in vals]
    g = ctx.gauss(x, P[0], P[1]); og = m.gauss(0, O[0], O[1])
    ex = ctx.exp(x, P[2]); oex = m.exp(0, O[2])
    po = ctx.poly(x, [P[3], P[4]]); opo = m.poly(0, [O[3], O[4]])
    root = ctx.add([g, ex, po], [P[5], P[6]]); m.add([og, oex, opo], [O[5], O[6]])
    return ctx, root, [x], m


@pytest.mark.parametrize("which", ["voigt", "mix3"])
def test_mixture_path_matches_stack_machine(gf, which):
    """An AddPdf of leaves is evaluated directly (P = sum c_k L_k) by default; the general
    stack machine gives the same NLL, gradient and per-event log P, and both match the
    oracle."""
    rng = np.random.default_rng(21)
    if which == "voigt":
        x = _voigt_data(300_007)
        a, ra, oa = pm.voigt_model(gf, nbins=2000)
        b, rb, ob = pm.voigt_model(gf, nbins=2000)
        m, free = om.voigt_model(nbins=2000)
        th = m.p[free] * np.array([1.0, 1.03, 0.95, 1.02, 1.05])
        p = m.p.copy(); p[free] = th
        cols = [x]
    else:
        a, ra, oa, m = _mix3_models(gf)
        b, rb, ob, _ = _mix3_models(gf)
        cols = [rng.uniform(-1.0, 2.0, 50_001)]
        th = m.p.copy()
        p = th
        free = np.arange(len(th))
    b.set_mixture_path(False)
    a.set_data(ra, oa, cols)
    b.set_data(rb, ob, cols)
    fa, ga = a.nll_grad(th)
    fb, gb = b.nll_grad(th)
    assert abs(fa - fb) <= 1e-12 * abs(fb)
    _grad_close(ga, gb, len(cols[0]), rel=1e-10)
    la, lb = a.logpdf(th), b.logpdf(th)
    per_event("mixture vs stack", la, lb, tol=2e-12)
    fo, go = m.nll(cols, p, grad=True)
    assert abs(fa - fo) <= 1e-9 * abs(fo)
    _grad_close(ga, go[free], len(cols[0]))
    lo_ = m.logpdf(cols, p)
    per_event("mixture vs oracle", la, lo_)


# ---- direct log-sum path (exponential / Gaussian leaves and their products) ------------------------
def _logsum_models(gf, which):
    """Returns (ctx_direct, ctx_stack, root_a, root_b, obs_a, obs_b, oracle model, columns)."""
    rng = np.random.default_rng(31)
    out = []
    for _ in range(2):
        ctx = gf.Context()
        m = oracle.Model1D([(0.0, 10.0)] if which == "exp" else [(0.0, 10.0), (-2.0, 3.0)])
        x = ctx.observable("x", 0.0, 10.0)
        y = ctx.observable("y", -2.0, 3.0)
        if which == "exp":
            a = ctx.parameter("a", -1.3, 0.1, -10, 10)
            root, obs = ctx.exp(x, a), [x]
            m.exp(0, m.param(-1.3))
        elif which == "gauss":
            mu = ctx.parameter("mu", 0.4, 0.1)
            s = ctx.parameter("s", 0.9, 0.1, 0.01, 5)
            root, obs = ctx.gauss(y, mu, s), [y]
            m = oracle.Model1D([(-2.0, 3.0)])
            m.gauss(0, m.param(0.4), m.param(0.9))
        else:  # exp(x) * gauss(y) * exp(y)-free: three leaves over two observables
            a = ctx.parameter("a", -0.7, 0.1, -10, 10)
            mu = ctx.parameter("mu", 0.4, 0.1)
            s = ctx.parameter("s", 0.9, 0.1, 0.01, 5)
            b = ctx.parameter("b", 0.2, 0.1, -10, 10, fixed=True)
            root = ctx.prod([ctx.exp(x, a), ctx.gauss(y, mu, s)])
            obs = [x, y]
            m.prod([m.exp(0, m.param(-0.7)), m.gauss(1, m.param(0.4), m.param(0.9))])
            m.param(0.2)
        out.append((ctx, root, obs, m))
    n = {"exp": 200_003, "gauss": 50_001, "prod": 100_001}[which]
    xs = synth.exp_events(n, -1.0, seed=4)
    xs[:5] = [0.0, 1e-30, 10.0, 5e-23, 2.0 ** -74]  # conversion path of the bit split
    ys = np.clip(rng.normal(0.4, 0.9, n), -2.0, 3.0)
    cols = {"exp": [xs], "gauss": [ys], "prod": [xs, ys]}[which]
    return out, cols


@pytest.mark.parametrize("which", ["exp", "gauss", "prod"])
def test_logsum_path_matches_stack_machine(gf, which):
    """A single exponential or Gaussian leaf, or a ProdPdf of them, runs on the direct
    log-sum kernel by default; the stack machine gives the same NLL and gradient, and both
    match the oracle."""
    ((a, ra, oa, m), (b, rb, ob, _)), cols = _logsum_models(gf, which)
    b.set_mixture_path(False)
    for n in (1, 2, 3, 257, len(cols[0])):
        cc = [c[:n] for c in cols]
        a.set_data(ra, oa, cc)
        b.set_data(rb, ob, cc)
        for scale in (1.0, 1.1):
            th = m.p[: len(a.free_params())] * scale
            fa, ga = a.nll_grad(th)
            fb, gb = b.nll_grad(th)
            assert abs(a.nll(th) - fa) <= 1e-12 * max(1.0, abs(fa))
            assert abs(fa - fb) <= 1e-11 * max(1.0, abs(fb)), (n, fa, fb)
            _grad_close(ga, gb, n, rel=1e-10)
            p = m.p.copy(); p[: len(th)] = th
            fo, go = m.nll(cc, p, grad=True)
            assert abs(fa - fo) <= 1e-9 * max(1.0, abs(fo))
            _grad_close(ga, go[: len(th)], n)


# ---- generic trees (Sec. 3: sums, products, nesting) ----------------------------------------------------
def _tree_models(gf):
    """Depth-3 tree over two observables: PROD(ADD(gauss, poly, exp), ADD(exp, gauss))."""
    ctx = gf.Context()
    m = oracle.Model1D([(-1.0, 2.0), (0.0, 3.0)])
    x = ctx.observable("x", -1.0, 2.0)
    y = ctx.observable("y", 0.0, 3.0)
    vals = [0.4, 0.6, 1.0, 0.3, 0.1, -0.7, 0.5, 0.2, -0.8, 1.5, 0.4, 0.35]
    names = ["mu", "s", "a0", "a1", "a2", "ax", "f1", "f2", "ay", "muy", "sy", "fy"]
    P = [ctx.parameter(nm, v, 0.01) for nm, v in zip(names, vals)]
    O = [m.param(v) for v in vals]
    g = ctx.gauss(x, P[0], P[1]); og = m.gauss(0, O[0], O[1])
    po = ctx.poly(x, [P[2], P[3], P[4]]); opo = m.poly(0, [O[2], O[3], O[4]])
    ex = ctx.exp(x, P[5]); oex = m.exp(0, O[5])
    a1 = ctx.add([g, po, ex], [P[6], P[7]]); oa1 = m.add([og, opo, oex], [O[6], O[7]])
    ey = ctx.exp(y, P[8]); oey = m.exp(1, O[8])
    gy = ctx.gauss(y, P[9], P[10]); ogy = m.gauss(1, O[9], O[10])
    a2 = ctx.add([ey, gy], [P[11]]); oa2 = m.add([oey, ogy], [O[11]])
    root = ctx.prod([a1, a2]); m.prod([oa1, oa2])
    return ctx, root, [x, y], m


@pytest.mark.parametrize("n", [7, 5001])
def test_nested_tree_parity(gf, n):
    ctx, root, obs, m = _tree_models(gf)
    rng = np.random.default_rng(3)
    xs = rng.uniform(-1, 2, n)
    ys = rng.uniform(0, 3, n)
    ctx.set_data(root, obs, [xs, ys])
    p = m.p.copy()
    lo_ = m.logpdf([xs, ys], p)
    lg = ctx.logpdf(p)
    per_event(f"nested tree n={n}", lg, lo_)
    f, g = ctx.nll_grad(p)
    fo, go = m.nll([xs, ys], p, grad=True)
    assert abs(f - fo) <= 1e-9 * abs(fo)
    _grad_close(g, go, n)


def test_product_of_exponentials_listing2(gf):
    ctx = gf.Context()
    x = ctx.observable("x", 0.0, 5.0)
    y = ctx.observable("y", 0.0, 5.0)
    ax = ctx.parameter("ax", -2.4, 0.1, -10, 10)
    ay = ctx.parameter("ay", -1.1, 0.1, -10, 10)
    root = ctx.prod([ctx.exp(x, ax), ctx.exp(y, ay)])
    xs = synth.exp_events(1000, -2.4, 0, 5, seed=1)
    ys = synth.exp_events(1000, -1.1, 0, 5, seed=2)
    ctx.set_data(root, [x, y], [xs, ys])
    m = oracle.Model1D([(0.0, 5.0), (0.0, 5.0)])
    m.prod([m.exp(0, m.param(-2.4)), m.exp(1, m.param(-1.1))])
    f, g = ctx.nll_grad(np.array([-2.4, -1.1]))
    fo, go = m.nll([xs, ys], grad=True)
    assert abs(f - fo) <= 1e-9 * abs(fo)
    _grad_close(g, go, 1000)


def test_densities_outside_float_range(gf):
    """Events whose density falls below 2^-80 (here x > ~7.2: P down to e^-76) are
    re-evaluated in FP64; the rest run in double-float pairs.  Both match the oracle."""
    ctx = gf.Context()
    x = ctx.observable("x", 0.0, 10.0)
    a1 = ctx.parameter("a1", -9.5, 0.1)
    a2 = ctx.parameter("a2", -8.0, 0.1)
    f = ctx.parameter("f", 0.3, 0.01)
    root = ctx.add([ctx.exp(x, a1), ctx.exp(x, a2)], [f])
    m = oracle.Model1D([(0.0, 10.0)])
    m.add([m.exp(0, m.param(-9.5)), m.exp(0, m.param(-8.0))], [m.param(0.3)])
    xs = np.random.default_rng(11).uniform(0.0, 10.0, 2001)
    ctx.set_data(root, [x], [xs])
    th = np.array([-9.5, -8.0, 0.3])
    lo_ = m.logpdf([xs], th)
    assert lo_.min() < -70 and (lo_ > -50).sum() > 500  # both regimes present
    lg = ctx.logpdf(th)
    per_event("outside float range", lg, lo_)
    fg, gg = ctx.nll_grad(th)
    fo, go = m.nll([xs], th, grad=True)
    assert abs(fg - fo) <= 1e-9 * abs(fo)
    _grad_close(gg, go, len(xs))


# ---- edge cases and errors --------------------------------------------------------------------------------
def test_nonfinite_is_reported(gf):
    # a polynomial that goes negative inside the range -> log P undefined
    ctx = gf.Context()
    x = ctx.observable("x", -1.0, 1.0)
    a0 = ctx.parameter("a0", 0.1, 0.01)
    a1 = ctx.parameter("a1", 1.0, 0.01)
    root = ctx.poly(x, [a0, a1])
    ctx.set_data(root, [x], [np.array([-0.9, 0.5, 0.2])])
    assert ctx.nll(np.array([0.1, 1.0])) == float("inf")


def test_out_of_range_events_rejected(gf):
    ctx, root, obs = pm.exp_model(gf)
    with pytest.raises(gf.GFError):
        ctx.set_data(root, obs, [np.array([1.0, 11.0])])


def test_device_columns_from_torch(gf):
    torch = pytest.importorskip("torch")
    x = synth.exp_events(10_001, -1.0)
    t = torch.tensor(x, dtype=torch.float64, device="cuda")
    ctx, root, obs = pm.exp_model(gf)
    ctx.set_data_device(root, obs, len(x), [t.data_ptr()], keep=t)
    m, free = om.exp_model(-1.3)
    assert abs(ctx.nll(np.array([-1.3])) - m.nll([x])) <= 1e-9 * abs(m.nll([x]))


def test_graph_replay_matches_direct_launches(gf):
    """Steady evaluations replay a captured CUDA graph; with graphs off the same kernels
    launch one by one.  Both give the same bits, for the NLL and the gradient."""
    lo, hi = synth.VOIGT_RANGE
    x = synth.voigt_threshold_events(100_003, **synth.VOIGT_TRUTH, lo=lo, hi=hi, seed=5)
    t = synth.VOIGT_TRUTH
    th0 = np.array([t["mu"], t["sigma"], t["width"], t["c"], t["frac"]])
    a, ra, oa = pm.voigt_model(gf, nbins=2000)
    b, rb, ob = pm.voigt_model(gf, nbins=2000)
    a.set_data(ra, oa, [x])
    b.set_data(rb, ob, [x])
    b.set_graphs(False)
    for k in range(4):
        th = th0 * (1.0 + 0.01 * k)
        fa, ga = a.nll_grad(th)
        rep, why = a.last_eval_graph()
        assert rep and why == ""
        fb, gb = b.nll_grad(th)
        assert b.last_eval_graph()[0] is False
        assert fa == fb and np.array_equal(ga, gb)
        assert a.nll(th) == b.nll(th)
