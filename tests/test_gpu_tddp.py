"""The time-dependent Dalitz model (Sec. 4: the D0 -> pi+ pi- pi0 mixing fit) on the
sm_103a path against the FP64 oracle.

Tolerances: per event |log P_gpu - log P_orc| <= 1e-12 max(1, kappa_i) (the interference
condition number of both amplitudes, (|a_NR| + sum |c_r a_r|)^2 / |A|^2 and the same for
B, the larger), 1e-9 relative on the NLL, gradients 1e-9 of their scale.  The full model
(free resonance masses and widths, the sigma_t density: 37 free parameters) is checked the
same way and fitted against the oracle's fit."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1311_1753_gb300 import synth
from tests import oracle_models as om
from tests import oracle_pool as op
from tests.parity import per_event

pytestmark = pytest.mark.gpu
SPEC = om.load_dalitz_spec()
TIME = dict(tau=0.41, x=0.01, y=0.007, scale=1.1)


@pytest.fixture(scope="module")
def gf():
    from paper_1311_1753_gb300 import gf as _gf
    return _gf


def _models(gf, nb=64, time=TIME):
    k = SPEC["kin"]
    d = oracle.Tddp(k["M"], k["m1"], k["m2"], k["m3"], k["R"], nb, nb)
    ctx = gf.Context()
    o12 = ctx.observable("s12", 0.0, 4.0)
    o13 = ctx.observable("s13", 0.0, 4.0)
    ot = ctx.observable("t", -2.0, 20.0)
    osg = ctx.observable("sigt", 0.0, 1.0)
    res = []
    for i, r in enumerate(SPEC["resonances"]):
        m0 = ctx.parameter(f"m0_{i}", r["m0"], 0.005, fixed=True)
        g0 = ctx.parameter(f"g0_{i}", r["g0"], 0.005, fixed=True)
        re = ctx.parameter(f"re_{i}", r["re"], 0.01)
        im = ctx.parameter(f"im_{i}", r["im"], 0.01)
        res.append(dict(channel=r["channel"], spin=r["spin"], mass=m0, width=g0, re=re, im=im))
        idx = [d.param(r[f]) for f in ("m0", "g0", "re", "im")]
        d.resonance(r["channel"], r["spin"], *idx)
    tp = [ctx.parameter(nm, v, 1e-3, 1e-3 if nm in ("tau", "scale") else -1.0,
                        5.0 if nm in ("tau", "scale") else 1.0) for nm, v in time.items()]
    d.time_params(*[d.param(v) for v in time.values()])
    root = ctx.tddp(o12, o13, ot, osg, k, res, *tp)
    ctx.set_norm_grid(root, nb, nb)
    return ctx, root, [o12, o13, ot, osg], d, np.array(ctx.free_params())


def _events(d, n, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    s12, s13 = synth.dalitz_events(n, om.dalitz_accept(om.dalitz_from_spec(SPEC), SPEC["envelope"]),
                                   seed=seed)
    sigt = rng.uniform(0.05, 0.15, n)
    t = np.clip(rng.exponential(0.41, n) + sigt * rng.standard_normal(n), -1.9, 19.0)
    return [s12, s13, t, sigt]


def _kappa(d, cols, p):
    s12, s13 = cols[0], cols[1]
    k = SPEC["kin"]
    s23 = k["M"] ** 2 + k["m1"] ** 2 + k["m2"] ** 2 + k["m3"] ** 2 - s12 - s13
    out = []
    for a, b in ((s12, s13), (s12, s23)):
        A = np.ones(len(a), complex)
        S = np.ones(len(a))
        for i, r in enumerate(SPEC["resonances"]):
            c = p[4 * i + 2] + 1j * p[4 * i + 3]
            v = c * d.amp(i, a, b, p=p)
            A += v
            S += np.abs(v)
        out.append(S ** 2 / np.abs(A) ** 2)
    return np.maximum(*out)


@pytest.mark.parametrize("n", [1, 257, 20_001])
def test_tddp_parity(gf, n):
    ctx, root, obs, d, free = _models(gf)
    cols = _events(d, n)
    ctx.set_data(root, obs, cols)
    rng = np.random.default_rng(1)
    for k in range(2):
        th = d.p[free] * (1 + (0.02 * rng.standard_normal(len(free)) if k else 0.0))
        p = d.p.copy(); p[free] = th
        lg = ctx.logpdf(th)
        lo_ = np.log(d.intensity_t(*cols, p=p)) - np.log(d.norm_t(p=p))
        per_event(f"tddp n={n}", lg, lo_, _kappa(d, cols, p))
        f, g = ctx.nll_grad(th)
        fo, go = d.nll_t(*cols, p=p, grad=True)
        assert abs(f - fo) <= 1e-9 * abs(fo)
        scale = np.abs(go[free]).max()
        assert np.all(np.abs(g - go[free]) <= 1e-9 * np.maximum(np.abs(go[free]), 1e-3 * scale)), (g, go[free])


def test_tddp_fit_matches_oracle_fit(gf):
    """A fit of the 16 coefficients, tau, x, y and the resolution scale (20 free) lands
    within 0.01 sigma of the oracle's fit from the same start."""
    from oracle import minimise
    ctx, root, obs, d, free = _models(gf, nb=48)
    cols = _events(d, 5000, seed=9)
    ctx.set_data(root, obs, cols)
    start = d.p[free] * (1 + 0.01 * np.random.default_rng(2).standard_normal(len(free)))
    for k, pid in enumerate(ctx.free_params()):
        ctx.set_value(pid, start[k])
    r = ctx.fit(tol=1e-9)
    assert r["status"] == gf.GF_OK

    def fg(q):
        p = d.p.copy(); p[free] = q
        f, g = d.nll_t(*cols, p=p, grad=True)
        return f, g[free]
    lo = np.array([-np.inf] * 16 + [1e-3, -1.0, -1.0, 1e-3])
    hi = np.array([np.inf] * 16 + [5.0, 1.0, 1.0, 5.0])
    lo[:16], hi[:16] = 0.0, 0.0  # unbounded
    ro = minimise.fit(fg, start, np.full(len(free), 1e-3), lo, hi, up=0.5, tol=1e-9)
    assert ro.converged
    assert np.all(np.abs(r["theta"] - ro.x) <= 0.01 * ro.err), np.max(np.abs(r["theta"] - ro.x) / ro.err)


def test_tddp_large_and_update(gf):
    """10^6 events (a size at which a 1D context would reorder its columns; the mixing
    context keeps the caller's order): sampled per-event log P against the oracle and the
    NLL equal to the sum of the stored log P.  gf_update_data then replaces the events,
    and rejects, with nothing replaced, events outside the kinematic region or with
    sigma_t <= 0."""
    ctx, root, obs, d, free = _models(gf)
    n = 1_000_000
    cols = _events(d, n, seed=11)
    ctx.set_data(root, obs, cols)
    th = d.p[free]
    lg = ctx.logpdf(th)
    idx = np.random.default_rng(5).choice(n, 300, replace=False)
    sub = [c[idx] for c in cols]
    lo_ = np.log(d.intensity_t(*sub, p=d.p)) - np.log(d.norm_t(p=d.p))
    per_event("tddp 1e6 sampled", lg[idx], lo_, _kappa(d, sub, d.p))
    f = ctx.nll(th)
    assert abs(f + np.sum(lg)) <= 1e-9 * abs(f)

    new = _events(d, n, seed=12)
    ctx.update_data(new)
    lg2 = ctx.logpdf(th)
    sub = [c[idx] for c in new]
    lo2 = np.log(d.intensity_t(*sub, p=d.p)) - np.log(d.norm_t(p=d.p))
    per_event("tddp 1e6 updated, sampled", lg2[idx], lo2, _kappa(d, sub, d.p))
    for k, v in ((3, 0.0), (0, 10.0)):
        bad = [c.copy() for c in cols]
        bad[k][n // 2] = v
        with pytest.raises(gf.GFError):
            ctx.update_data(bad)
        assert np.array_equal(ctx.logpdf(th), lg2)


def test_tddp_parity_strong_mixing(gf):
    """x = 0.2, y = 0.15, sigma scale 0.6: every mixing term (cosh, cos, sinh, sin) and the
    reflection of the smeared exponentials weighs in; per-event log P, NLL and gradient
    against the oracle."""
    ctx, root, obs, d, free = _models(gf, time=dict(tau=0.41, x=0.2, y=0.15, scale=0.6))
    cols = _events(d, 4099, seed=21)
    ctx.set_data(root, obs, cols)
    p = d.p
    lg = ctx.logpdf(p[free])
    lo_ = np.log(d.intensity_t(*cols, p=p)) - np.log(d.norm_t(p=p))
    per_event("tddp strong mixing", lg, lo_, _kappa(d, cols, p))
    f, g = ctx.nll_grad(p[free])
    fo, go = d.nll_t(*cols, p=p, grad=True)
    assert abs(f - fo) <= 1e-9 * abs(fo)
    scale = np.abs(go[free]).max()
    assert np.all(np.abs(g - go[free]) <= 1e-9 * np.maximum(np.abs(go[free]), 1e-3 * scale)), (g, go[free])



# ---- the full mixing model: free resonance shapes and the sigma_t density ------------------
DENS = (2.3, 0.4, -0.3)
SIGT = (0.02, 0.5)


def _full_models(gf, nb=48, time=TIME, dens=DENS):
    """Masses and widths of resonances 0..6 free (resonance 7 fixed, as in the free-shape Dalitz fit), the 16
    coefficients, tau, x, y, scale and the sigma_t density's b0, b1, b2: 37 free."""
    k = SPEC["kin"]
    d = om.tddp_from_spec(SPEC, nb, time, dens, SIGT)
    ctx = gf.Context()
    o12 = ctx.observable("s12", 0.0, 4.0)
    o13 = ctx.observable("s13", 0.0, 4.0)
    ot = ctx.observable("t", -2.0, 20.0)
    osg = ctx.observable("sigt", *SIGT)
    res = []
    nres = len(SPEC["resonances"])
    for i, r in enumerate(SPEC["resonances"]):
        fixed = i == nres - 1
        m0 = ctx.parameter(f"m0_{i}", r["m0"], 0.005, 0.4, 1.75, fixed=fixed)
        g0 = ctx.parameter(f"g0_{i}", r["g0"], 0.005, 0.01, 0.6, fixed=fixed)
        re = ctx.parameter(f"re_{i}", r["re"], 0.01)
        im = ctx.parameter(f"im_{i}", r["im"], 0.01)
        res.append(dict(channel=r["channel"], spin=r["spin"], mass=m0, width=g0, re=re, im=im))
    tp = [ctx.parameter(nm, v, 1e-3, 1e-3 if nm in ("tau", "scale") else -1.0,
                        5.0 if nm in ("tau", "scale") else 1.0) for nm, v in time.items()]
    bs = [ctx.parameter(f"b{j}", v, 0.01) for j, v in enumerate(dens)]
    root = ctx.tddp(o12, o13, ot, osg, k, res, *tp)
    ctx.tddp_sigt_density(root, *bs)
    ctx.set_norm_grid(root, nb, nb)
    free = np.array([q for q in range(len(d.p)) if not (q in (4 * (nres - 1), 4 * (nres - 1) + 1))])
    assert len(free) == len(ctx.free_params()) == 37
    return ctx, root, [o12, o13, ot, osg], d, free


def _full_events(n, seed, dens=DENS):
    """(s12, s13) from the Dalitz density, sigma_t from the Gamma(2) density at each point
    (truncated to its range), t from the smeared exponential."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s12, s13 = synth.dalitz_events(n, om.dalitz_accept(om.dalitz_from_spec(SPEC), SPEC["envelope"]),
                                   seed=seed)
    k = SPEC["kin"]
    sc = (k["M"] ** 2 + k["m1"] ** 2 + k["m2"] ** 2 + k["m3"] ** 2) / 3
    lam = np.exp(dens[0] + dens[1] * (s12 - sc) + dens[2] * (s13 - sc))
    sigt = np.empty(n)
    todo = np.arange(n)
    while len(todo):
        v = rng.gamma(2.0, 1.0 / lam[todo])
        ok = (v > SIGT[0]) & (v < SIGT[1])
        sigt[todo[ok]] = v[ok]
        todo = todo[~ok]
    t = np.clip(rng.exponential(0.41, n) + 1.1 * sigt * rng.standard_normal(n), -1.9, 19.0)
    return [s12, s13, t, sigt]


@pytest.mark.parametrize("n", [1, 257, 20_001])
def test_tddp_full_model_parity(gf, n):
    ctx, root, obs, d, free = _full_models(gf)
    cols = _full_events(n, seed=31)
    ctx.set_data(root, obs, cols)
    rng = np.random.default_rng(7)
    for k in range(2):
        p = d.p.copy()
        if k:
            p[free] *= 1 + 0.01 * rng.standard_normal(len(free))
        th = p[free]
        lg = ctx.logpdf(th)
        lo_ = (np.log(d.intensity_t(*cols, p=p)) - np.log(d.norm_t(p=p)) +
               d.sigt_logd(cols[0], cols[1], cols[3], p))
        per_event(f"tddp full n={n}", lg, lo_, _kappa(d, cols, p))
        f, g = ctx.nll_grad(th)
        fo, go = (op.tddp_nll(SPEC, 48, TIME, DENS, p, cols, grad=True) if n > 1000 else
                  d.nll_t(*cols, p=p, grad=True))
        assert abs(f - fo) <= 1e-9 * abs(fo), (f, fo)
        scale = np.abs(go[free]).max()
        assert np.all(np.abs(g - go[free]) <= 1e-9 * np.maximum(np.abs(go[free]), 1e-3 * scale)), \
            (np.abs(g - go[free]) / np.maximum(np.abs(go[free]), 1e-3 * scale)).max()
        assert abs(ctx.nll(th) - f) <= 1e-12 * abs(f)


def test_tddp_full_model_fit_matches_oracle_fit(gf):
    """The paper's mixing fit has about 40 free parameters: here 37 (16 coefficients, 14
    masses and widths, tau, x, y, the resolution scale, the sigma_t density's 3), fitted
    on 10^4 events from a displaced start, within 0.01 sigma of the oracle's fit."""
    from oracle import minimise
    ctx, root, obs, d, free = _full_models(gf)
    cols = _full_events(10_000, seed=41)
    ctx.set_data(root, obs, cols)
    start = d.p[free] * (1 + 0.003 * np.random.default_rng(3).standard_normal(len(free)))
    for k, pid in enumerate(ctx.free_params()):
        ctx.set_value(pid, start[k])
    r = ctx.fit(tol=1e-8)
    assert r["status"] == gf.GF_OK, r

    def fg(q):
        p = d.p.copy()
        p[free] = q
        f, g = op.tddp_nll(SPEC, 48, TIME, DENS, p, cols, grad=True)
        return f, g[free]
    names = [q % 4 for q in free[:30]]
    lo = np.array([0.4 if m == 0 else 0.01 if m == 1 else 0.0 for m in names] +
                  [1e-3, -1.0, -1.0, 1e-3, 0.0, 0.0, 0.0])
    hi = np.array([1.75 if m == 0 else 0.6 if m == 1 else 0.0 for m in names] +
                  [5.0, 1.0, 1.0, 5.0, 0.0, 0.0, 0.0])
    step = np.array([0.005 if m < 2 else 0.01 for m in names] + [1e-3] * 4 + [0.01] * 3)
    ro = minimise.fit(fg, start, step, lo, hi, up=0.5, tol=1e-8)
    assert ro.converged
    dev = (r["theta"] - ro.x) / ro.err
    from tests.parity import WORST
    WORST["tddp full fit (37 free, 1e4 events): max |theta - theta_orc| / sigma"] = float(np.abs(dev).max())
    assert np.all(np.abs(dev) <= 0.01), dev
