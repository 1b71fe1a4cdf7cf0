"""ConvolutionPdf and the relativistic Breit-Wigner line shape on the sm_103a path against
the FP64 oracle (Sec. 3: ConvolutionPdf; Sec. 4: the binned D*+ line-width fit, a P-wave
relativistic Breit-Wigner convolved with a resolution of several Gaussians).

Tolerances: |log P_gpu - log P_orc| <= 1e-12 per event, 1e-9 relative on the NLL or
metric, gradients 1e-9 of their scale; fitted parameters within 0.01 sigma."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import minimise
from paper_1311_1753_gb300 import synth

from tests.parity import per_event

pytestmark = pytest.mark.gpu
LO, HI = synth.VOIGT_RANGE
D0, PIC = 1.86484, 0.13957
RW = 0.002  # resolution support [-RW, RW]


@pytest.fixture(scope="module")
def gf():
    from paper_1311_1753_gb300 import gf as _gf
    return _gf


def _grad_close(g, go, rel=1e-9):
    scale = np.abs(go).max()
    assert np.all(np.abs(g - go) <= rel * np.maximum(np.abs(go), 1e-3 * scale) + 1e-12 * scale), (g, go)


def _data(n, seed=7):
    """n events of the 1D composite workload above the D0 pi+ threshold (the line shape
    vanishes below it: such events would have P = 0)."""
    x = synth.voigt_threshold_events(n + n // 50 + 10, **synth.VOIGT_TRUTH, lo=LO, hi=HI,
                                     seed=seed)
    return x[x > PIC][:n]


# parameter values in declaration order (theta of every free one, in this order)
BW = [0.14543, 8.3e-5, D0, D0, PIC, 1.5]          # dm0, gamma0, shift, ma, mb, R
RES3 = [0.0, 2.0e-4, 0.0, 4.5e-4, 1.0e-4, 9.0e-4, 0.6, 0.3]  # 3 Gaussians + 2 fractions
BKG = [LO, 0.5, 20.0, 0.35]                        # threshold x0, power, c; signal fraction


def zach_models(gf, nbins=4000, lattice=860, with_bkg=True, model="relbw"):
    """(relbw or Voigtian) x (3 Gaussians) [+ threshold background], GPU and oracle."""
    ctx = gf.Context()
    x = ctx.observable("dm", LO, HI)
    r = ctx.observable("res", -RW, RW)
    m = oracle.Model1D([(LO, HI), (-RW, RW)], nbins=nbins)
    if model == "relbw":
        names = ["dm0", "g0", "shift", "ma", "mb", "R"]
        fixed = [False, False, True, True, True, True]
        P = [ctx.parameter(nm, v, 1e-5, fixed=f) for nm, v, f in zip(names, BW, fixed)]
        O = [m.param(v) for v in BW]
        sig = ctx.relbw(x, *P, spin=1)
        osig = m.relbw(0, *O, spin=1)
    else:
        P = [ctx.parameter("mu", 0.1455, 1e-5), ctx.parameter("s", 1e-4, 1e-5),
             ctx.parameter("G", 8e-5, 1e-5)]
        O = [m.param(0.1455), m.param(1e-4), m.param(8e-5)]
        sig = ctx.voigt(x, *P)
        osig = m.voigt(0, *O)
    ctx.set_norm_grid(sig, nbins)
    # the three means fixed: widths and fractions free (at most 8 free parameters in a
    # convolution's model and resolution together)
    Q = [ctx.parameter(f"r{k}", v, 1e-5, fixed=(k in (0, 2, 4))) for k, v in enumerate(RES3)]
    OQ = [m.param(v) for v in RES3]
    g = [ctx.gauss(r, Q[2 * k], Q[2 * k + 1]) for k in range(2)]
    g.append(ctx.gauss(r, Q[4], Q[5]))
    og = [m.gauss(1, OQ[2 * k], OQ[2 * k + 1]) for k in range(2)]
    og.append(m.gauss(1, OQ[4], OQ[5]))
    res = ctx.add(g, [Q[6], Q[7]])
    ores = m.add(og, [OQ[6], OQ[7]])
    conv = ctx.conv(x, sig, res, lattice)
    oconv = m.conv(0, osig, ores, lattice)
    root, oroot = conv, oconv
    if with_bkg:
        B = [ctx.parameter(nm, v, 1e-3, fixed=(k < 2)) for k, (nm, v) in
             enumerate(zip(["x0", "pw", "c", "f"], BKG))]
        OB = [m.param(v) for v in BKG]
        th = ctx.threshold(x, B[0], B[1], B[2])
        ctx.set_norm_grid(th, nbins)
        root = ctx.add([conv, th], [B[3]])
        oroot = m.add([oconv, m.threshold(0, OB[0], OB[1], OB[2])], [OB[3]])
    free = [pid for pid in ctx.free_params()]
    return ctx, root, [x], m, np.array(free)


def _theta(ctx, m, free, scale=None):
    th = m.p[free].copy()
    if scale is not None:
        th *= scale[: len(th)]
    p = m.p.copy()
    p[free] = th
    return th, p


@pytest.mark.parametrize("n", [1, 1001, 100_003])
def test_relbw_leaf_parity(gf, n):
    ctx = gf.Context()
    x = ctx.observable("dm", LO, HI)
    fixed = [False, False, True, True, True, True]
    P = [ctx.parameter(f"p{k}", v, 1e-5, fixed=f) for k, (v, f) in enumerate(zip(BW, fixed))]
    root = ctx.relbw(x, *P, spin=1)
    ctx.set_norm_grid(root, 4000)
    xs = _data(n)
    ctx.set_data(root, [x], [xs])
    m = oracle.Model1D([(LO, HI)], nbins=4000)
    m.relbw(0, *[m.param(v) for v in BW], spin=1)
    for sc in (1.0, 1.0003):
        th = np.array([BW[0] * sc, BW[1] * (2 - sc)])
        p = m.p.copy(); p[:2] = th
        lg, lo_ = ctx.logpdf(th), m.logpdf([xs], p)
        per_event("relbw leaf", lg, lo_)
        f, g = ctx.nll_grad(th)
        fo, go = m.nll([xs], p, grad=True)
        assert abs(f - fo) <= 1e-9 * abs(fo)
        _grad_close(g, go[:2])
    # at and below threshold the density is zero on both sides
    below = np.array([LO, PIC - 1e-9, PIC - 1e-13])
    ctx.set_data(root, [x], [below])
    assert np.all(np.isneginf(ctx.logpdf(th))) and np.all(np.isneginf(m.logpdf([below], p)))


@pytest.mark.parametrize("model", ["relbw", "voigt"])
@pytest.mark.parametrize("n", [1, 1001, 50_001])
def test_conv_unbinned_parity(gf, model, n):
    ctx, root, obs, m, free = zach_models(gf, nbins=2000, lattice=430, model=model)
    xs = _data(n, seed=11)
    ctx.set_data(root, obs, [xs])
    for sc in (None, np.array([1.0001, 0.97, 1.02, 1.03, 0.98, 1.05, 0.97, 1.04, 1.01, 0.99])):
        th, p = _theta(ctx, m, free, sc)
        lg, lo_ = ctx.logpdf(th), m.logpdf([xs], p)
        per_event(f"conv {model}", lg, lo_)
        f, g = ctx.nll_grad(th)
        fo, go = m.nll([xs], p, grad=True)
        assert abs(f - fo) <= 1e-9 * abs(fo)
        _grad_close(g, go[free])


@pytest.mark.parametrize("metric", [0, 1, 2])
def test_conv_binned_parity(gf, metric):
    ctx, root, obs, m, free = zach_models(gf)
    counts, edges = np.histogram(_data(1_000_000, seed=13), 4000, (LO, HI))
    c = 0.5 * (edges[1:] + edges[:-1])
    n = counts.astype(float)
    ctx.set_binned_data(root, obs, [4000], n)
    ctx.set_metric(metric)
    K = n.sum() * (HI - LO) / 4000
    th, p = _theta(ctx, m, free, np.array([1.00005, 1.1, 0.95, 1.05, 0.9, 1.1, 1.02, 0.97, 1.03]))
    f, g = ctx.nll_grad(th)
    fo, go = m.binned([c], n, K, metric, s2=np.maximum(n, 1.0), p=p, grad=True)
    assert abs(f - fo) <= 1e-9 * abs(fo)
    _grad_close(g, go[free])
    # the same with graphs off: the same bits
    ctx.set_graphs(False)
    f2, g2 = ctx.nll_grad(th)
    assert f2 == f and np.array_equal(g2, g)


def test_zach_binned_chisq_fit_matches_oracle(gf):
    """The paper's binned D*+ fit shape (P-wave relativistic Breit-Wigner convolved with
    three Gaussians, plus a threshold background) fitted by chi-squared on 4000 bins:
    gf_fit lands within 0.01 sigma of the oracle's BFGS fit."""
    ctx, root, obs, m, free = zach_models(gf)
    counts, edges = np.histogram(_data(2_000_000, seed=17), 4000, (LO, HI))
    c = 0.5 * (edges[1:] + edges[:-1])
    n = counts.astype(float)
    ctx.set_binned_data(root, obs, [4000], n)
    ctx.set_metric(gf.GF_METRIC_CHISQ)
    # fit the line (dm0, gamma0), the core resolution width and the signal fraction;
    # the other resolution parameters stay at their values
    keep = {0, 1, 2, 8}
    for k, pid in enumerate(ctx.free_params()):
        if k not in keep:
            ctx.set_fixed(pid, True)
    sub = np.array(sorted(keep))
    free2 = free[sub]
    start = m.p[free2] * np.array([1.00003, 1.2, 0.9, 0.95])
    for k, pid in enumerate(ctx.free_params()):
        ctx.set_value(pid, start[k])
    r = ctx.fit(tol=1e-9)
    assert r["status"] == gf.GF_OK
    K = n.sum() * (HI - LO) / 4000
    s2 = np.maximum(n, 1.0)

    def fg(q):
        p = m.p.copy(); p[free2] = q
        f, g = m.binned([c], n, K, 2, s2=s2, p=p, grad=True)
        return f, g[free2]
    ro = minimise.fit(fg, start, np.array([1e-5, 1e-5, 1e-5, 1e-3]), up=1.0, tol=1e-9)
    assert ro.converged
    assert np.all(np.abs(r["theta"] - ro.x) <= 0.01 * ro.err), (r["theta"], ro.x, ro.err)
    assert np.all(np.abs(r["err"] / ro.err - 1) < 0.01)


def test_conv_rejections(gf):
    ctx = gf.Context()
    x = ctx.observable("dm", LO, HI)
    r = ctx.observable("res", -RW, RW)
    y = ctx.observable("y", 0.0, 1.0)
    mu, s = ctx.parameter("mu", 0.1455, 1e-5), ctx.parameter("s", 1e-4, 1e-5)
    z0, z1 = ctx.parameter("z0", 0.0, 1e-5, fixed=True), ctx.parameter("z1", 3e-4, 1e-5)
    sig = ctx.gauss(x, mu, s)
    res = ctx.gauss(r, z0, z1)
    conv = ctx.conv(x, sig, res)
    with pytest.raises(gf.GFError):
        ctx.conv(x, conv, res)  # nested
    bad = ctx.conv(x, sig, ctx.prod([ctx.gauss(r, z0, z1), ctx.gauss(y, z0, z1)]))
    with pytest.raises(gf.GFError):  # resolution over two observables
        ctx.set_data(bad, [x, y], [_data(10), np.full(10, 0.5)])
        ctx.nll(np.array([0.1455, 1e-4, 3e-4]))
    with pytest.raises(gf.GFError):  # a free shift of the line shape
        c2 = gf.Context()
        xx = c2.observable("dm", LO, HI)
        P = [c2.parameter(f"p{k}", v, 1e-5) for k, v in enumerate(BW)]
        rb = c2.relbw(xx, *P)
        c2.set_data(rb, [xx], [_data(10)])
