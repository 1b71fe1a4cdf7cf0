"""Oracle-side builders for the workloads (tests only)."""
from __future__ import annotations

import json
import os

import numpy as np

import oracle
from paper_1311_1753_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def exp_model(alpha=-1.0, lo=0.0, hi=10.0):
    """The truncated exponential e^{alpha x} on [0, 10] (Listing 1)."""
    m = oracle.Model1D([(lo, hi)])
    a = m.param(alpha)
    m.exp(0, a)
    return m, [a]


def voigt_model(truth=None, nbins=10000):
    """The line-shape fit: frac * Voigt(mu, sigma, width) + (1-frac) * threshold(x0, power, c).
    Returns (model, free parameter indices in the order mu, sigma, width, c, frac)."""
    t = dict(synth.VOIGT_TRUTH if truth is None else truth)
    m = oracle.Model1D([synth.VOIGT_RANGE], nbins=nbins)
    mu, s, w = m.param(t["mu"]), m.param(t["sigma"]), m.param(t["width"])
    x0, pw, c = m.param(t["x0"]), m.param(t["power"]), m.param(t["c"])
    f = m.param(t["frac"])
    v = m.voigt(0, mu, s, w)
    b = m.threshold(0, x0, pw, c)
    m.add([v, b], [f])
    return m, [mu, s, w, c, f]


def dalitz_model_file(seed=synth.SEED_DALITZ_MODEL):
    return os.path.join(GOLDEN, f"dalitz_model_{seed}.json")


def load_dalitz_spec(seed=synth.SEED_DALITZ_MODEL):
    with open(dalitz_model_file(seed)) as fh:
        return json.load(fh)


def dalitz_from_spec(spec, nbx=512, nby=512):
    """Oracle Dalitz model with parameter order, per resonance r:
    m0_r, g0_r, re_r, im_r  (index 4 r + k)."""
    k = spec["kin"]
    d = oracle.Dalitz(k["M"], k["m1"], k["m2"], k["m3"], k["R"], nbx, nby)
    for r in spec["resonances"]:
        i0 = d.param(r["m0"])
        i1 = d.param(r["g0"])
        i2 = d.param(r["re"])
        i3 = d.param(r["im"])
        d.resonance(r["channel"], r["spin"], i0, i1, i2, i3)
    return d


def dalitz_accept(d, envelope):
    def acc(s12, s13, u):
        inside = d.inside(s12, s13)
        out = np.zeros(len(s12), dtype=bool)
        idx = np.nonzero(inside)[0]
        if len(idx):
            P = d.intensity(s12[idx], s13[idx])
            out[idx] = u[idx] * envelope < P
        return out
    return acc


def tddp_from_spec(spec, nb, time, dens=None, sigt_range=(0.02, 0.5)):
    """Oracle time-dependent Dalitz model: per resonance r the parameters m0_r, g0_r, re_r,
    im_r (index 4 r + k), then tau, x, y, scale, then (with dens) b0, b1, b2."""
    k = spec["kin"]
    d = oracle.Tddp(k["M"], k["m1"], k["m2"], k["m3"], k["R"], nb, nb)
    for r in spec["resonances"]:
        idx = [d.param(r[f]) for f in ("m0", "g0", "re", "im")]
        d.resonance(r["channel"], r["spin"], *idx)
    tp = [d.param(v) for v in (time["tau"], time["x"], time["y"], time["scale"])]
    if dens is None:
        d.time_params(*tp)
    else:
        d.time_params(*tp, density=tuple(d.param(v) for v in dens), sigt_range=sigt_range)
    return d
