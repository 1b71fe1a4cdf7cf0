"""Fits through gf_fit (the library's BFGS on the GPU likelihood) against the oracle's
own BFGS on the oracle likelihood: fitted values within 0.01 sigma of the oracle's, and
errors within 1 %."""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle
from oracle import minimise
from paper_1311_1753_gb300 import synth
from tests import oracle_models as om
from tests import product_models as pm

pytestmark = pytest.mark.gpu
SPEC = om.load_dalitz_spec()


@pytest.fixture(scope="module")
def gf():
    from paper_1311_1753_gb300 import gf as _gf
    return _gf


def _oracle_fit(m, free, cols, x0, step, lo, hi, fun=None):
    def fg(x):
        p = m.p.copy()
        p[free] = x
        f, g = (fun or (lambda q: m.nll(cols, q, grad=True)))(p)
        return f, g[free]
    return minimise.fit(fg, x0, step, lo, hi, tol=1e-10)


@pytest.mark.parametrize("use_grad", [True, False])
def test_exponential_fit(gf, use_grad):
    x = synth.exp_events(100_000, -1.0)
    ctx, root, obs = pm.exp_model(gf, -2.0)
    ctx.set_data(root, obs, [x])
    r = ctx.fit(tol=1e-10, use_grad=use_grad)
    assert r["status"] == gf.GF_OK
    m, free = om.exp_model(-2.0)
    o = _oracle_fit(m, free, [x], np.array([-2.0]), np.array([0.1]), np.array([-10.0]),
                    np.array([10.0]))
    assert o.converged
    assert abs(r["theta"][0] - o.x[0]) <= 0.01 * o.err[0]
    assert abs(r["err"][0] / o.err[0] - 1) < 0.01
    # and the stationarity root of the exponential MLE (quadrature)
    mean = x.mean()
    g = lambda a: integrate.quad(lambda t: t * math.exp(a * t), 0, 10)[0] / \
        integrate.quad(lambda t: math.exp(a * t), 0, 10)[0] - mean
    root_ = optimize.brentq(g, -1.5, -0.5, xtol=1e-14)
    assert abs(r["theta"][0] - root_) <= 0.01 * o.err[0]


def test_voigt_fit(gf):
    lo, hi = synth.VOIGT_RANGE
    x = synth.voigt_threshold_events(200_000, **synth.VOIGT_TRUTH, lo=lo, hi=hi, seed=99)
    m, free = om.voigt_model(nbins=2000)
    truth = m.p[free]
    start = truth * np.array([1.0002, 1.1, 0.85, 1.1, 0.93])
    ctx, root, obs = pm.voigt_model(gf, nbins=2000)
    for k, pid in enumerate(ctx.free_params()):
        ctx.set_value(pid, start[k])
    ctx.set_data(root, obs, [x])
    r = ctx.fit(tol=1e-9)
    assert r["status"] == gf.GF_OK, r
    step = np.array([1e-5, 1e-5, 1e-5, 0.5, 0.01])
    lo_b = np.array([0.143, 1e-5, 1e-6, 0.0, 0.0])
    hi_b = np.array([0.148, 2e-3, 1e-3, 200.0, 1.0])
    o = _oracle_fit(m, free, [x], start, step, lo_b, hi_b)
    assert o.converged
    assert np.all(np.abs(r["theta"] - o.x) <= 0.01 * o.err), (r["theta"] - o.x) / o.err
    assert np.all(np.abs(r["err"] / o.err - 1) < 0.01)


def test_dalitz_fixed_shape_fit_small_grid(gf):
    nres = len(SPEC["resonances"])
    d = om.dalitz_from_spec(SPEC, 128, 128)
    d_full = om.dalitz_from_spec(SPEC)
    s12, s13 = synth.dalitz_events(20_000, om.dalitz_accept(d_full, SPEC["envelope"]), seed=77)
    free = [4 * r + k for r in range(nres) for k in (2, 3)]
    truth = d.p[free]
    rng = np.random.default_rng(4)
    start = truth + 0.02 * rng.standard_normal(len(truth))
    ctx, root, obs = pm.dalitz_model(gf, SPEC, nbx=128, nby=128)
    for k, pid in enumerate(ctx.free_params()):
        ctx.set_value(pid, start[k])
    ctx.set_data(root, obs, [s12, s13])
    r = ctx.fit(tol=1e-9)
    assert r["status"] == gf.GF_OK, r
    o = _oracle_fit(d, free, None, start, np.full(len(free), 0.01), np.zeros(len(free)),
                    np.zeros(len(free)), fun=lambda q: d.nll(s12, s13, q, grad=True))
    assert o.converged
    assert np.all(np.abs(r["theta"] - o.x) <= 0.01 * o.err), (r["theta"] - o.x) / o.err
    assert np.all(np.abs(r["err"] / o.err - 1) < 0.01)


def test_autograd_wrapper(gf):
    torch = pytest.importorskip("torch")
    from paper_1311_1753_gb300.autograd import nll
    x = synth.exp_events(50_000, -1.0)
    ctx, root, obs = pm.exp_model(gf)
    ctx.set_data(root, obs, [x])
    th = torch.tensor([-1.3], dtype=torch.float64, requires_grad=True)
    f = nll(ctx, th)
    f.backward()
    m, _ = om.exp_model(-1.3)
    fo, go = m.nll([x], grad=True)
    assert abs(f.item() - fo) <= 1e-9 * abs(fo)
    assert abs(th.grad.item() - go[0]) <= 1e-9 * abs(go[0])


def test_dalitz_free_shape_mixed_fit_small(gf):
    """The free-shape Dalitz model: 30 free parameters (7 masses and widths free), FP32 amplitudes with
    FP64 sums and normalisation, fused gradient; against the oracle's FP64 fit."""
    nres = len(SPEC["resonances"])
    d = om.dalitz_from_spec(SPEC, 128, 128)
    d_full = om.dalitz_from_spec(SPEC)
    s12, s13 = synth.dalitz_events(20_000, om.dalitz_accept(d_full, SPEC["envelope"]), seed=78)
    free = []
    for r in range(nres):
        if r != nres - 1:
            free += [4 * r, 4 * r + 1]
        free += [4 * r + 2, 4 * r + 3]
    truth = d.p[free]
    rng = np.random.default_rng(5)
    start = truth * (1 + 0.01 * rng.standard_normal(len(truth)))
    ctx, root, obs = pm.dalitz_model(gf, SPEC, precision=gf.GF_MIXED, free_shapes=True, nbx=128,
                                     nby=128)
    for k, pid in enumerate(ctx.free_params()):
        ctx.set_value(pid, start[k])
    ctx.set_data(root, obs, [s12, s13])
    r = ctx.fit(tol=1e-8)  # FP32 BFGS to EDM 1e-4, then the FP64 refinement to 1e-8
    step = np.array([0.005 if k % 4 < 2 else 0.01 for k in free])
    lo_b = np.array([0.4 if k % 4 == 0 else 0.01 if k % 4 == 1 else 0.0 for k in free])
    hi_b = np.array([1.75 if k % 4 == 0 else 0.6 if k % 4 == 1 else 0.0 for k in free])
    o = _oracle_fit(d, free, None, start, step, lo_b, hi_b,
                    fun=lambda q: d.nll(s12, s13, q, grad=True))
    assert o.converged
    dev = (r["theta"] - o.x) / o.err
    print("mixed fit: status", r["status"], "edm", r["edm"], "calls", r["n_calls"],
          "max |dev|/sigma", np.abs(dev).max())
    assert np.all(np.abs(dev) <= 0.01), dev
    assert np.all(np.abs(r["err"] / o.err - 1) < 0.02)
