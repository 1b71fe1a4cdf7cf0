"""gf_nll_noalloc, the entry point for callers that cannot call cudaMalloc (device memory
owned by a pool or framework that grants no extra buffers, or a device footprint that
must not grow once running): same NLL as gf_nll, computed with the library's static
scratch array and no allocation.  Checked against gf_nll on two calls in a row, for a
grid-normalised tree (Voigtian + threshold), an analytic one (exponential), nested sums
and products in the linear and log domains; and its refusals (shared observables in a
product, Dalitz nodes, oversized trees, a capturing stream).

Collected last on purpose: it must pass alone in a fresh process and after every other
test."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1311_1753_gb300 import synth
from tests import product_models as pm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    from paper_1311_1753_gb300 import gf as _gf
    return _gf


def _check(gf, torch, build, x, thetas):
    cols = x if isinstance(x, list) else [x]
    # reference: the allocating path (gf_set_data + gf_nll)
    ref_ctx, ref_root, ref_obs = build()
    ref_ctx.set_data(ref_root, ref_obs, cols)
    # allocation-free path: a context holding only the model, caller-owned buffers
    ctx, root, obs = build()
    xd = [torch.tensor(c, dtype=torch.float64, device="cuda") for c in cols]
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for th in thetas:  # two calls in a row, different theta
        ctx.nll_noalloc(root, obs, len(cols[0]), [c.data_ptr() for c in xd], th,
                        out.data_ptr())
        torch.cuda.synchronize()
        got = out.item()
        want = ref_ctx.nll(th)
        assert np.isfinite(got)
        assert abs(got - want) <= 1e-12 * abs(want), (got, want)


def test_noalloc_matches_gf_nll_voigt(gf):
    torch = pytest.importorskip("torch")
    lo, hi = synth.VOIGT_RANGE
    x = synth.voigt_threshold_events(300_001, **synth.VOIGT_TRUTH, lo=lo, hi=hi, seed=4321)
    t = synth.VOIGT_TRUTH
    th0 = np.array([t["mu"], t["sigma"], t["width"], t["c"], t["frac"]])
    _check(gf, torch, lambda: pm.voigt_model(gf), x,
           [th0, th0 * np.array([1.00001, 1.03, 0.95, 1.05, 0.97])])


def test_noalloc_matches_gf_nll_exponential(gf):
    torch = pytest.importorskip("torch")
    x = synth.exp_events(100_003, -1.0, seed=99)
    _check(gf, torch, lambda: pm.exp_model(gf), x, [np.array([-1.0]), np.array([-1.7])])


def test_noalloc_rejects_sizes_beyond_its_scratch(gf):
    torch = pytest.importorskip("torch")
    ctx, root, obs = pm.voigt_model(gf, nbins=200_000)  # 2 x 200,000 bins > 262,144
    x = torch.full((16,), 0.15, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    t = synth.VOIGT_TRUTH
    th = np.array([t["mu"], t["sigma"], t["width"], t["c"], t["frac"]])
    with pytest.raises(gf.GFError) as e:
        ctx.nll_noalloc(root, obs, 16, [x.data_ptr()], th, out.data_ptr())
    assert e.value.code == gf.GF_EINVAL and "262,144" in str(e.value)


def _two_obs_model(gf, kind):
    """Trees over x in [0, 10] and y in [-1, 3]:
    nested  AddPdf(ProdPdf(exp(x), gauss(y)), ProdPdf(poly(x), threshold(y)))
    logprod ProdPdf(exp(x), gauss(y))                     (log domain)
    linprod ProdPdf(poly(x), threshold(y))                (linear domain)
    addadd  AddPdf(AddPdf(gauss(x), exp(x)), poly(x))     (nested sums, one observable)"""
    ctx = gf.Context(0, gf.GF_FP64)
    x = ctx.observable("x", 0.0, 10.0)
    y = ctx.observable("y", -1.0, 3.0)
    a = ctx.parameter("a", -0.3, 0.05, -5.0, 5.0)
    mu = ctx.parameter("mu", 1.0, 0.05, -1.0, 3.0)
    sg = ctx.parameter("sg", 0.7, 0.05, 0.05, 5.0)
    c0 = ctx.parameter("c0", 1.0, 0.1, fixed=True)
    c1 = ctx.parameter("c1", 0.2, 0.02, 0.0, 2.0)
    x0 = ctx.parameter("x0", -1.0, 0.1, fixed=True)
    pw = ctx.parameter("pw", 0.5, 0.1, fixed=True)
    cc = ctx.parameter("cc", 1.5, 0.1, 0.0, 20.0)
    f1 = ctx.parameter("f1", 0.4, 0.02, 0.0, 1.0)
    if kind == "nested":
        root = ctx.add([ctx.prod([ctx.exp(x, a), ctx.gauss(y, mu, sg)]),
                        ctx.prod([ctx.poly(x, [c0, c1]), ctx.threshold(y, x0, pw, cc)])], [f1])
        return ctx, root, [x, y]
    if kind == "logprod":
        return ctx, ctx.prod([ctx.exp(x, a), ctx.gauss(y, mu, sg)]), [x, y]
    if kind == "linprod":
        return ctx, ctx.prod([ctx.poly(x, [c0, c1]), ctx.threshold(y, x0, pw, cc)]), [x, y]
    f2 = ctx.parameter("f2", 0.3, 0.02, 0.0, 1.0)
    inner = ctx.add([ctx.gauss(x, ctx.parameter("mx", 4.0, 0.1, 0.0, 10.0), sg), ctx.exp(x, a)],
                    [f1])
    return ctx, ctx.add([inner, ctx.poly(x, [c0, c1])], [f2]), [x]


def _free_theta(ctx):
    return np.array([ctx.value(p) for p in ctx.free_params()])


@pytest.mark.parametrize("kind", ["nested", "logprod", "linprod", "addadd"])
def test_noalloc_matches_gf_nll_nested_trees(gf, kind):
    torch = pytest.importorskip("torch")
    rng = np.random.Generator(np.random.PCG64(77))
    n = 200_003
    x = rng.uniform(0.0, 10.0, n)
    y = -1.0 + rng.gamma(1.5, 0.6, n)
    y = np.where(y < 3.0, y, rng.uniform(-1.0, 3.0, n))
    ctx, root, obs = _two_obs_model(gf, kind)
    th0 = _free_theta(ctx)
    cols = [x, y] if len(obs) == 2 else x
    _check(gf, torch, lambda: _two_obs_model(gf, kind), cols,
           [th0, th0 * (1.0 + 0.03 * np.cos(np.arange(len(th0))))])


def test_noalloc_rejects_unsupported_trees(gf):
    torch = pytest.importorskip("torch")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    col = torch.full((8,), 0.5, dtype=torch.float64, device="cuda")
    # a product whose factors share an observable
    ctx = gf.Context(0, gf.GF_FP64)
    x = ctx.observable("x", 0.0, 1.0)
    a = ctx.parameter("a", -1.0, 0.1)
    root = ctx.prod([ctx.exp(x, a), ctx.exp(x, a)])
    with pytest.raises(gf.GFError) as e:
        ctx.nll_noalloc(root, [x], 8, [col.data_ptr()], np.array([-1.0]), out.data_ptr())
    assert e.value.code == gf.GF_EINVAL and "share an observable" in str(e.value)
    # more than 32 instructions: an AddPdf of 8 leaves inside an AddPdf of 2 (8 leaves,
    # 10 scales, 8 additions + 2 leaves ... beyond the program's size)
    ctx = gf.Context(0, gf.GF_FP64)
    x = ctx.observable("x", 0.0, 1.0)
    f = ctx.parameter("f", 0.1, 0.01, fixed=True)
    a = ctx.parameter("a", -1.0, 0.1)
    leaves = [ctx.exp(x, a) for _ in range(8)]
    big = ctx.add([ctx.add(leaves, [f] * 7), ctx.add([ctx.exp(x, a) for _ in range(4)], [f] * 3)],
                  [f])
    with pytest.raises(gf.GFError) as e:
        ctx.nll_noalloc(big, [x], 8, [col.data_ptr()], np.array([-1.0]), out.data_ptr())
    assert e.value.code == gf.GF_EINVAL and "32 instructions" in str(e.value)
    # a Dalitz node
    from tests import oracle_models as om
    spec = om.load_dalitz_spec()
    dctx, droot, dobs = pm.dalitz_model(gf, spec)
    th = np.array([dctx.value(p) for p in dctx.free_params()])
    with pytest.raises(gf.GFError) as e:
        dctx.nll_noalloc(droot, dobs, 8, [col.data_ptr(), col.data_ptr()], th, out.data_ptr())
    assert e.value.code == gf.GF_EINVAL and "unsupported node" in str(e.value)


def test_noalloc_refuses_a_capturing_stream(gf):
    """The call stages theta from host stack memory, which a graph cannot replay: on a
    stream that is capturing it must return GF_EINVAL and queue nothing (the capture
    then ends cleanly, with an empty graph)."""
    torch = pytest.importorskip("torch")
    ctx, root, obs = pm.exp_model(gf)
    x = torch.tensor(synth.exp_events(1000, -1.0, seed=5), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    ctx.set_stream(s.cuda_stream)
    g = torch.cuda.CUDAGraph()
    with pytest.raises(gf.GFError) as e:
        with torch.cuda.graph(g, stream=s):
            ctx.nll_noalloc(root, obs, 1000, [x.data_ptr()], np.array([-1.0]), out.data_ptr())
    assert e.value.code == gf.GF_EINVAL and "capturing" in str(e.value)
    torch.cuda.synchronize()
    # the context still works outside the capture
    ctx.nll_noalloc(root, obs, 1000, [x.data_ptr()], np.array([-1.0]), out.data_ptr())
    torch.cuda.synchronize()
    assert np.isfinite(out.item())
