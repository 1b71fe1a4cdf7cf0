"""Builders of the workloads through the library's C ABI (tests only).  Parameter
creation order matches tests/oracle_models.py so theta vectors line up."""
from __future__ import annotations

from paper_1311_1753_gb300 import synth


def exp_model(gf, alpha=-2.0, precision=None, lo=0.0, hi=10.0):
    """The truncated exponential of Listing 1: alpha in [-10, 10], step 0.1."""
    ctx = gf.Context(0, gf.GF_FP64 if precision is None else precision)
    x = ctx.observable("x", lo, hi)
    a = ctx.parameter("alpha", alpha, 0.1, -10.0, 10.0)
    root = ctx.exp(x, a)
    return ctx, root, [x]


def voigt_model(gf, truth=None, precision=None, nbins=10000, free_shape=False, width_lo=1e-6):
    """Voigtian + threshold background (the line-shape fit); free mu, sigma, width, c,
    frac."""
    t = dict(synth.VOIGT_TRUTH if truth is None else truth)
    lo, hi = synth.VOIGT_RANGE
    ctx = gf.Context(0, gf.GF_FP64 if precision is None else precision)
    x = ctx.observable("dm", lo, hi)
    mu = ctx.parameter("mu", t["mu"], 1e-5, 0.143, 0.148)
    s = ctx.parameter("sigma", t["sigma"], 1e-5, 1e-5, 2e-3)
    w = ctx.parameter("width", t["width"], 1e-5, width_lo, 1e-3)
    x0 = ctx.parameter("x0", t["x0"], 1e-4, fixed=not free_shape)
    pw = ctx.parameter("power", t["power"], 0.01, fixed=not free_shape)
    c = ctx.parameter("c", t["c"], 0.5, 0.0, 200.0)
    f = ctx.parameter("frac", t["frac"], 0.01, 0.0, 1.0)
    v = ctx.voigt(x, mu, s, w)
    b = ctx.threshold(x, x0, pw, c)
    if nbins != 10000:
        ctx.set_norm_grid(v, nbins)
        ctx.set_norm_grid(b, nbins)
    root = ctx.add([v, b], [f])
    return ctx, root, [x]


def dalitz_model(gf, spec, precision=None, free_shapes=False, nbx=512, nby=512, fixed_last=True):
    """The eight-resonance Dalitz models: resonance r has parameters m0_r, g0_r, re_r, im_r (index 4r + k).
    free_shapes: masses and widths free (except the last resonance if fixed_last)."""
    k = spec["kin"]
    ctx = gf.Context(0, gf.GF_FP64 if precision is None else precision)
    o12 = ctx.observable("s12", 0.0, 4.0)
    o13 = ctx.observable("s13", 0.0, 4.0)
    res = []
    nres = len(spec["resonances"])
    for i, r in enumerate(spec["resonances"]):
        shape_free = free_shapes and not (fixed_last and i == nres - 1)
        m0 = ctx.parameter(f"m0_{i}", r["m0"], 0.005, 0.4, 1.75, fixed=not shape_free)
        g0 = ctx.parameter(f"g0_{i}", r["g0"], 0.005, 0.01, 0.6, fixed=not shape_free)
        re = ctx.parameter(f"re_{i}", r["re"], 0.01)
        im = ctx.parameter(f"im_{i}", r["im"], 0.01)
        res.append(dict(channel=r["channel"], spin=r["spin"], mass=m0, width=g0, re=re, im=im))
    root = ctx.dalitz(o12, o13, k, res)
    if (nbx, nby) != (512, 512):
        ctx.set_norm_grid(root, nbx, nby)
    return ctx, root, [o12, o13]
