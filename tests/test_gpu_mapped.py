"""MappedPdf and CompositePdf (Sec. 3) on the sm_103a path against the FP64 oracle.

Tolerances: |log P_gpu - log P_orc| <= 1e-12 per event, 1e-9 relative on the NLL or
metric, gradients 1e-9 of their scale."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1311_1753_gb300 import synth

from tests.parity import per_event

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    from paper_1311_1753_gb300 import gf as _gf
    return _gf


def _grad_close(g, go, rel=1e-9):
    scale = np.abs(go).max()
    assert np.all(np.abs(g - go) <= rel * np.maximum(np.abs(go), 1e-3 * scale) + 1e-12 * scale), (g, go)


def mapped_models(gf, nb=4000):
    """Gaussian on [0, 1.7), exponential on [1.7, 3.2), linear polynomial on [3.2, 5]."""
    ctx = gf.Context()
    x = ctx.observable("x", 0.0, 5.0)
    m = oracle.Model1D([(0.0, 5.0)], nbins=nb)
    vals = [1.0, 0.8, -0.6, 1.0, 0.3, 1.7, 3.2]
    fixed = [False, False, False, True, False, True, True]
    P = [ctx.parameter(f"p{k}", v, 0.01, fixed=f) for k, (v, f) in enumerate(zip(vals, fixed))]
    O = [m.param(v) for v in vals]
    node = ctx.mapped(x, [ctx.gauss(x, P[0], P[1]), ctx.exp(x, P[2]), ctx.poly(x, [P[3], P[4]])],
                      [P[5], P[6]])
    ctx.set_norm_grid(node, nb)
    m.mapped(0, [m.gauss(0, O[0], O[1]), m.exp(0, O[2]), m.poly(0, [O[3], O[4]])], [O[5], O[6]])
    return ctx, node, [x], m, np.array(ctx.free_params())


def composite_models(gf, nb=4000, shell="gauss"):
    """shell(core(x)): core a quadratic polynomial in x, shell Gaussian or exponential;
    plus an AddPdf with an exponential so that the node sits inside a larger tree."""
    ctx = gf.Context()
    x = ctx.observable("x", 0.0, 5.0)
    u = ctx.observable("u", -50.0, 50.0)
    m = oracle.Model1D([(0.0, 5.0), (-50.0, 50.0)], nbins=nb)
    vals = [0.2, 0.9, -0.05, 1.0, 1.5, -0.3, 0.6]
    P = [ctx.parameter(f"p{k}", v, 0.01) for k, v in enumerate(vals)]
    O = [m.param(v) for v in vals]
    core = ctx.poly(x, [P[0], P[1], P[2]])
    ocore = m.poly(0, [O[0], O[1], O[2]])
    if shell == "gauss":
        sh, osh = ctx.gauss(u, P[3], P[4]), m.gauss(1, O[3], O[4])
    else:
        sh, osh = ctx.exp(u, P[5]), m.exp(1, O[5])
    comp = ctx.composite(x, core, sh)
    ctx.set_norm_grid(comp, nb)
    ocomp = m.composite(0, ocore, osh)
    root = ctx.add([comp, ctx.exp(x, P[5])], [P[6]])
    m.add([ocomp, m.exp(0, O[5])], [O[6]])
    free = np.array(ctx.free_params())
    return ctx, root, [x], m, free


@pytest.mark.parametrize("which", ["mapped", "composite-gauss", "composite-exp"])
@pytest.mark.parametrize("n", [1, 999, 60_001])
def test_parity_unbinned(gf, which, n):
    if which == "mapped":
        ctx, root, obs, m, free = mapped_models(gf)
    else:
        ctx, root, obs, m, free = composite_models(gf, shell=which.split("-")[1])
    xs = synth.exp_events(n + 3, -0.5, 0.0, 5.0, seed=3)[:n]
    if n > 3:
        xs[:3] = [1.7, 3.2, 5.0]  # on the boundaries and the top of the range
    ctx.set_data(root, obs, [xs])
    for sc in (1.0, 1.03):
        th = m.p[free] * sc
        p = m.p.copy(); p[free] = th
        lg, lo_ = ctx.logpdf(th), m.logpdf([xs], p)
        per_event("mapped/composite", lg, lo_)
        f, g = ctx.nll_grad(th)
        fo, go = m.nll([xs], p, grad=True)
        assert abs(f - fo) <= 1e-9 * max(1.0, abs(fo))
        _grad_close(g, go[free])


@pytest.mark.parametrize("metric", [1, 2])
def test_parity_binned(gf, metric):
    ctx, root, obs, m, free = mapped_models(gf)
    x = synth.exp_events(200_000, -0.5, 0.0, 5.0, seed=8)
    counts, edges = np.histogram(x, 500, (0.0, 5.0))
    c = 0.5 * (edges[1:] + edges[:-1])
    n = counts.astype(float)
    ctx.set_binned_data(root, obs, [500], n)
    ctx.set_metric(metric)
    th = m.p[free] * 1.02
    p = m.p.copy(); p[free] = th
    f, g = ctx.nll_grad(th)
    fo, go = m.binned([c], n, n.sum() * 0.01, metric, s2=np.maximum(n, 1.0), p=p, grad=True)
    assert abs(f - fo) <= 1e-9 * abs(fo)
    _grad_close(g, go[free])


def test_rejections(gf):
    ctx = gf.Context()
    x = ctx.observable("x", 0.0, 5.0)
    a = ctx.parameter("a", -0.5, 0.1)
    b = ctx.parameter("b", 2.0, 0.1)  # a free boundary: refused
    node = ctx.mapped(x, [ctx.exp(x, a), ctx.exp(x, a)], [b])
    with pytest.raises(gf.GFError):
        ctx.set_data(node, [x], [np.array([1.0, 3.0])])
    with pytest.raises(gf.GFError):  # a Voigtian shell: refused at declaration
        mu, s, w = (ctx.parameter(nm, v, 0.1) for nm, v in (("mu", 1), ("s", 1), ("w", 1)))
        ctx.composite(x, ctx.exp(x, a), ctx.voigt(x, mu, s, w))
