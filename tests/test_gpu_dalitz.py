"""Parity of the sm_103a Dalitz path with the FP64 oracle (fixed-shape and free-shape eight-resonance models).

Per event: |log P_gpu - log P_orc| <= 1e-12 max(1, kappa_i) for every event, with the
interference condition number kappa_i = (|a_NR| + sum_r |c_r A_r|)^2 / |A|^2.  Total NLL
1e-9 relative; gradients 1e-9 relative to their scale.  FP32 (mixed) results: errors are
measured and bounded (per event: median 1e-5, 99th percentile 1e-3 relative; NLL 1e-6
relative).  The full-size cases (10^6 events with fixed shapes, 5 x 10^6 with free masses and widths) compare
every event; the oracle runs over the host cores there (tests/oracle_pool.py)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1311_1753_gb300 import synth
from tests import oracle_models as om
from tests import oracle_pool as op
from tests import product_models as pm
from tests.parity import WORST, per_event

pytestmark = pytest.mark.gpu

SPEC = om.load_dalitz_spec()


@pytest.fixture(scope="module")
def gf():
    from paper_1311_1753_gb300 import gf as _gf
    return _gf


_cache = {}


def _events(n, seed=synth.SEED_DALITZ_EVENTS):
    key = (n, seed)
    if key not in _cache:
        acc = op.dalitz_accept(SPEC) if n > 100_000 else om.dalitz_accept(
            om.dalitz_from_spec(SPEC), SPEC["envelope"])
        _cache[key] = synth.dalitz_events(n, acc, seed)
    return _cache[key]


def _theta_all(spec):
    out = []
    for r in spec["resonances"]:
        out += [r["m0"], r["g0"], r["re"], r["im"]]
    return np.array(out)


def _free_idx(nres, free_shapes, fixed_last=True):
    idx = []
    for r in range(nres):
        if free_shapes and not (fixed_last and r == nres - 1):
            idx += [4 * r, 4 * r + 1]
        idx += [4 * r + 2, 4 * r + 3]
    return idx


@pytest.mark.parametrize("n", [1, 31, 33, 5000])
@pytest.mark.parametrize("free_shapes", [False, True])
def test_dalitz_fp64_parity(gf, n, free_shapes):
    s12, s13 = _events(5000)
    s12, s13 = s12[:n], s13[:n]
    nres = len(SPEC["resonances"])
    ctx, root, obs = pm.dalitz_model(gf, SPEC, free_shapes=free_shapes)
    ctx.set_data(root, obs, [s12, s13])
    d = om.dalitz_from_spec(SPEC)
    p = _theta_all(SPEC)
    free = _free_idx(nres, free_shapes)
    rng = np.random.default_rng(11)
    for trial in range(2):
        q = p.copy()
        if trial:
            q[free] *= 1 + 0.03 * rng.standard_normal(len(free))
        th = q[free]
        lg = ctx.logpdf(th)
        P, kap = d.intensity(s12, s13, q, kappa=True)
        N, _ = d.norm(q)
        per_event(f"dalitz fp64 n={n} free_shapes={free_shapes}", lg, np.log(P / N), kap)
        f, g = ctx.nll_grad(th)
        fo, go = d.nll(s12, s13, q, grad=True)
        assert abs(f - fo) <= 1e-9 * max(1.0, abs(fo)), (f, fo)
        go = go[free]
        scale = np.maximum(np.abs(go), 1e-6 * max(n, 1))
        assert np.all(np.abs(g - go) <= 1e-9 * scale + 1e-9 * np.abs(go).max()), (g, go)


def test_dalitz_gram_matches_oracle_norm(gf):
    nres = len(SPEC["resonances"])
    ctx, root, obs = pm.dalitz_model(gf, SPEC)
    s12, s13 = _events(100)
    ctx.set_data(root, obs, [s12, s13])
    th = _theta_all(SPEC)[_free_idx(nres, False)]
    G = ctx.dalitz_gram(th, nres)
    assert np.allclose(G, G.conj().T, rtol=0, atol=1e-12 * np.abs(G).max())
    c = np.concatenate([[1.0], th[0::2] + 1j * th[1::2]])
    N = (c.conj() @ G @ c).real
    d = om.dalitz_from_spec(SPEC)
    No, cnt = d.norm()
    assert cnt == 155812
    assert abs(N / No - 1) < 1e-12
    # diagonal = per-resonance integrals of |A_r|^2 (fit-fraction denominators)
    for r, res in enumerate(SPEC["resonances"]):
        assert abs(G[r + 1, r + 1].real / res["G_rr"] - 1) < 1e-12


def test_dalitz_full_size(gf):
    """10^6 events (fixed shapes) in the benchmark's launch shape: NLL against the oracle's
    full sum, and log P of every event within 1e-12 max(1, kappa_i)."""
    nres = len(SPEC["resonances"])
    s12, s13 = _events(1_000_000)
    ctx, root, obs = pm.dalitz_model(gf, SPEC)
    ctx.set_data(root, obs, [s12, s13])
    d = om.dalitz_from_spec(SPEC)
    p = _theta_all(SPEC)
    th = p[_free_idx(nres, False)]
    f = ctx.nll(th)
    fo = op.dalitz_nll(SPEC, p, s12, s13)
    assert abs(f - fo) <= 1e-9 * abs(fo)
    P, kap = op.dalitz_intensity(SPEC, p, s12, s13, kappa=True)
    N, _ = d.norm(p)
    per_event("dalitz fixed full 1e6", ctx.logpdf(th), np.log(P / N), kap)
    WORST["dalitz fixed full 1e6: events with kappa > 1e3"] = float((kap > 1e3).sum())


def test_free_shape_full_size_fp64_and_mixed(gf):
    """5 x 10^6 events, 30 free parameters (masses and widths of 7 resonances free), the
    512 x 512 grid: the FP64 plan against the oracle on every event, NLL and gradient;
    the mixed plan (FP32 amplitudes) with its error percentiles stated and bounded."""
    nres = len(SPEC["resonances"])
    s12, s13 = _events(5_000_000, synth.SEED_DALITZ_BIG)
    d = om.dalitz_from_spec(SPEC)
    p = _theta_all(SPEC)
    free = _free_idx(nres, True)
    q = p.copy()
    q[free] *= 1 + 0.01 * np.random.default_rng(12).standard_normal(len(free))
    th = q[free]
    P, kap = op.dalitz_intensity(SPEC, q, s12, s13, kappa=True)
    N, _ = d.norm(q)
    lo_ = np.log(P / N)
    fo, go = op.dalitz_nll(SPEC, q, s12, s13, grad=True)
    go = go[free]
    ctx, root, obs = pm.dalitz_model(gf, SPEC, free_shapes=True)
    ctx.set_data(root, obs, [s12, s13])
    per_event("dalitz free fp64 full 5e6", ctx.logpdf(th), lo_, kap)
    f, g = ctx.nll_grad(th)
    assert abs(f - fo) <= 1e-9 * abs(fo), (f, fo)
    scale = np.maximum(np.abs(go), 1e-6 * len(s12))
    assert np.all(np.abs(g - go) <= 1e-9 * scale + 1e-9 * np.abs(go).max()), (g, go)
    ctx.close()
    mctx, mroot, mobs = pm.dalitz_model(gf, SPEC, precision=gf.GF_MIXED, free_shapes=True)
    mctx.set_data(mroot, mobs, [s12, s13])
    rel = np.abs(np.expm1(mctx.logpdf(th) - lo_))
    pct = {q_: float(np.quantile(rel, q_)) for q_ in (0.5, 0.9, 0.99, 0.999)}
    pct[1.0] = float(rel.max())
    for q_, v in pct.items():
        WORST[f"dalitz free mixed full 5e6: per-event |P/P_orc - 1| quantile {q_}"] = v
    assert pct[0.5] < 1e-5 and pct[0.99] < 1e-3
    fm, gm = mctx.nll_grad(th)
    WORST["dalitz free mixed full 5e6: NLL relative error"] = abs(fm / fo - 1)
    WORST["dalitz free mixed full 5e6: max |dgrad| / max |grad|"] = float(
        np.max(np.abs(gm - go)) / np.abs(go).max())
    assert abs(fm - fo) <= 1e-6 * abs(fo)
    assert np.max(np.abs(gm - go)) <= 1e-3 * np.abs(go).max()


def test_dalitz_mixed_precision_errors(gf):
    nres = len(SPEC["resonances"])
    s12, s13 = _events(5000)
    d = om.dalitz_from_spec(SPEC)
    p = _theta_all(SPEC)
    free = _free_idx(nres, True)
    ctx, root, obs = pm.dalitz_model(gf, SPEC, precision=gf.GF_MIXED, free_shapes=True)
    ctx.set_data(root, obs, [s12, s13])
    th = p[free]
    lg = ctx.logpdf(th)
    P = d.intensity(s12, s13, p)
    N, _ = d.norm(p)
    rel = np.abs(np.expm1(lg - np.log(P / N)))
    assert np.median(rel) < 1e-5 and np.quantile(rel, 0.99) < 1e-3
    f, g = ctx.nll_grad(th)
    fo, go = d.nll(s12, s13, p, grad=True)
    assert abs(f - fo) <= 1e-6 * abs(fo)
    go = go[free]
    assert np.max(np.abs(g - go)) <= 1e-3 * np.abs(go).max() + 1e-2
