"""gf_prefetch_data: the next events (up to two sets ahead) copied and range-checked on the
library's copy stream while the current ones are evaluated, then loaded by gf_update_data
as a swap of device buffer sets (Sec. 2's data loading, pipelined with the evaluation).

The loaded set must give exactly what a fresh gf_set_data of the same events in the
caller's order gives (the same kernels: bitwise), per event against the oracle, in both
buffer sets and after alternating them, also when the loaded set was re-sorted (its
second evaluation) while the next one was being copied; a range error in a prefetched set
is reported by the loading call and leaves the loaded set in place."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1311_1753_gb300 import synth
from tests import oracle_models as om
from tests import product_models as pm
from tests.parity import per_event

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    from paper_1311_1753_gb300 import gf as _gf
    return _gf


def _voigt_data(n, seed):
    lo, hi = synth.VOIGT_RANGE
    return synth.voigt_threshold_events(n, **synth.VOIGT_TRUTH, lo=lo, hi=hi, seed=seed)


def _ptrs(cols):
    return [c.ctypes.data for c in cols]


def _fresh(gf, x, sort=True):
    ctx, root, obs = pm.voigt_model(gf, nbins=2000)
    ctx.set_event_sort(sort)
    ctx.set_data(root, obs, [x])
    return ctx


def test_prefetched_sets_match_a_fresh_load(gf):
    n = 400_003
    xs = [np.ascontiguousarray(_voigt_data(n, synth.SEED_VOIGT + 200 + k)) for k in range(3)]
    m, free = om.voigt_model(nbins=2000)
    th = m.p[free] * np.array([1.0, 1.02, 0.97, 1.01, 0.99])
    p = m.p.copy()
    p[free] = th
    ctx, root, obs = pm.voigt_model(gf, nbins=2000)
    ctx.set_data(root, obs, [xs[0]])
    ctx.nll_grad(th)
    ref = {}
    for k in (1, 2):
        f = _fresh(gf, xs[k], sort=False)
        ref[k] = f.nll_grad(th)
        f.close()
    # load 1, 2, 1, 2: each prefetched while the previous set is evaluated (its second
    # evaluation: the loaded set is sorted again meanwhile)
    for step, k in enumerate((1, 2, 1, 2)):
        ctx.prefetch_data_ptrs(n, _ptrs([xs[k]]))
        ctx.nll_grad(th)
        ctx.update_data_ptrs(n, _ptrs([xs[k]]))
        f, g = ctx.nll_grad(th)
        assert f == ref[k][0] and np.array_equal(g, ref[k][1]), (step, f, ref[k][0])
        assert ctx.last_eval_graph()[0]
    per_event("prefetched set", ctx.logpdf(th), m.logpdf([xs[2]], p))
    fo, go = m.nll([xs[2]], p, grad=True)
    assert abs(ref[2][0] - fo) <= 1e-9 * abs(fo)
    ctx.close()


def test_two_prefetches_in_flight(gf):
    """Two sets staged ahead (three device buffer sets in rotation), loaded in order, each
    equal to a fresh load; a third prefetch while two wait drops the oldest, and loading
    the newer of two pending sets drops the older one."""
    n = 200_001
    xs = [np.ascontiguousarray(_voigt_data(n, synth.SEED_VOIGT + 400 + k)) for k in range(6)]
    m, free = om.voigt_model(nbins=2000)
    th = m.p[free] * np.array([1.0, 0.99, 1.03, 0.98, 1.01])
    ref = {}
    for k in range(6):
        f = _fresh(gf, xs[k], sort=False)
        ref[k] = f.nll_grad(th)
        f.close()
    ctx, root, obs = pm.voigt_model(gf, nbins=2000)
    ctx.set_data(root, obs, [xs[0]])
    ctx.prefetch_data_ptrs(n, _ptrs([xs[1]]))
    ctx.prefetch_data_ptrs(n, _ptrs([xs[2]]))
    order = [1, 2, 3, 4, 5, 1, 2, 3]
    for step, k in enumerate(order):
        f, g = ctx.nll_grad(th)  # the loaded set, while the next two are copied
        ctx.update_data_ptrs(n, _ptrs([xs[k]]))
        if step + 2 < len(order):
            ctx.prefetch_data_ptrs(n, _ptrs([xs[order[step + 2]]]))
        f, g = ctx.nll_grad(th)
        assert f == ref[k][0] and np.array_equal(g, ref[k][1]), (step, k)
    # a full queue (2 and 3 wait): staging 4 drops 2; loading 4 then drops 3
    ctx.prefetch_data_ptrs(n, _ptrs([xs[2]]))
    ctx.prefetch_data_ptrs(n, _ptrs([xs[3]]))
    ctx.prefetch_data_ptrs(n, _ptrs([xs[4]]))
    ctx.update_data_ptrs(n, _ptrs([xs[4]]))
    f, g = ctx.nll_grad(th)
    assert f == ref[4][0] and np.array_equal(g, ref[4][1])
    # 3 was dropped: loading it copies it on the spot
    ctx.update_data_ptrs(n, _ptrs([xs[3]]))
    f, g = ctx.nll_grad(th)
    assert f == ref[3][0] and np.array_equal(g, ref[3][1])
    ctx.close()


def test_started_evaluation_with_loads_in_between(gf):
    """gf_nll_grad_start / gf_nll_grad_finish: the same bits as gf_nll_grad, also with the
    next set loaded and a later one prefetched while the started evaluation runs (it keeps
    the events it started with); a second start, an evaluation or a new data set while
    one is in flight, and a finish without a start, are refused."""
    n = 150_001
    xs = [np.ascontiguousarray(_voigt_data(n, synth.SEED_VOIGT + 500 + k)) for k in range(5)]
    m, free = om.voigt_model(nbins=2000)
    th = m.p[free] * np.array([1.0, 1.01, 0.98, 1.02, 0.99])
    ref = {}
    for k in range(5):
        f = _fresh(gf, xs[k], sort=False)
        ref[k] = f.nll_grad(th)
        f.close()
    ctx, root, obs = pm.voigt_model(gf, nbins=2000)
    ctx.set_event_sort(False)
    ctx.set_data(root, obs, [xs[0]])
    ctx.nll_grad_start(th)
    with pytest.raises(gf.GFError):
        ctx.nll_grad_start(th)
    with pytest.raises(gf.GFError):
        ctx.nll(th)
    with pytest.raises(gf.GFError):
        ctx.set_data(root, obs, [xs[1]])
    f, g = ctx.nll_grad_finish()
    assert f == ref[0][0] and np.array_equal(g, ref[0][1])
    with pytest.raises(gf.GFError):
        ctx.nll_grad_finish()
    ctx.prefetch_data_ptrs(n, _ptrs([xs[1]]))
    ctx.prefetch_data_ptrs(n, _ptrs([xs[2]]))
    for k in range(4):
        ctx.nll_grad_start(th)
        ctx.update_data_ptrs(n, _ptrs([xs[k + 1]]))
        if k + 3 < 5:
            ctx.prefetch_data_ptrs(n, _ptrs([xs[k + 3]]))
        f, g = ctx.nll_grad_finish()
        assert f == ref[k][0] and np.array_equal(g, ref[k][1]), k
    f, g = ctx.nll_grad(th)
    assert f == ref[4][0] and np.array_equal(g, ref[4][1])
    ctx.close()


def test_prefetch_range_error_keeps_the_loaded_set(gf):
    n = 50_001
    x = np.ascontiguousarray(_voigt_data(n, synth.SEED_VOIGT + 300))
    bad = x.copy()
    bad[n // 3] = synth.VOIGT_RANGE[1] + 1.0
    ctx, root, obs = pm.voigt_model(gf, nbins=2000)
    ctx.set_data(root, obs, [x])
    t = synth.VOIGT_TRUTH
    th = np.array([t["mu"], t["sigma"], t["width"], t["c"], t["frac"]])
    f0 = ctx.nll(th)
    ctx.prefetch_data_ptrs(n, _ptrs([bad]))
    with pytest.raises(gf.GFError):
        ctx.update_data_ptrs(n, _ptrs([bad]))
    assert ctx.nll(th) == f0
    # a prefetched set loaded under other pointers: dropped, the plain copy path runs
    y = np.ascontiguousarray(_voigt_data(n, synth.SEED_VOIGT + 301))
    ctx.prefetch_data_ptrs(n, _ptrs([y]))
    y2 = y.copy()
    ctx.update_data([y2])
    f1 = ctx.nll(th)
    ref = _fresh(gf, y)
    assert abs(f1 - ref.nll(th)) <= 1e-12 * abs(f1)
    ref.close()
    ctx.close()


def test_prefetch_without_sorting_and_refusals(gf):
    """An exponential (no Voigtian: nothing to sort) takes the prefetch too; a context
    without data and a Dalitz data set are refused."""
    n = 100_000
    rng = np.random.default_rng(5)
    a, b = (np.ascontiguousarray(rng.exponential(1.0, n) % 10.0) for _ in range(2))
    th = np.array([-1.3])
    ctx, root, obs = pm.exp_model(gf)
    ctx.set_data(root, obs, [a])
    ctx.prefetch_data_ptrs(n, _ptrs([b]))
    ctx.update_data_ptrs(n, _ptrs([b]))
    f = ctx.nll(th)
    ref, rroot, robs = pm.exp_model(gf)
    ref.set_data(rroot, robs, [b])
    assert f == ref.nll(th)
    ref.close()
    ctx.close()
    empty = gf.Context()
    empty.observable("x", 0.0, 1.0)
    with pytest.raises(gf.GFError):
        empty.prefetch_data_ptrs(1, _ptrs([np.zeros(1)]))
    empty.close()
    spec = om.load_dalitz_spec()
    dz, droot, dobs = pm.dalitz_model(gf, spec, nbx=64, nby=64)
    d = om.dalitz_from_spec(spec, 64, 64)
    rng = np.random.default_rng(7)
    s12, s13 = [], []
    while len(s12) < 10:
        u, v = rng.uniform(0.0, 3.5, 2)
        if d.inside(np.array([u]), np.array([v]))[0]:
            s12.append(u)
            s13.append(v)
    cols = [np.array(s12), np.array(s13)]
    dz.set_data(droot, dobs, cols)
    with pytest.raises(gf.GFError):
        dz.prefetch_data_ptrs(10, _ptrs(cols))
    dz.close()
