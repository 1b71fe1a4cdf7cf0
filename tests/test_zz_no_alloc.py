"""gf_nll_noalloc, the entry point for callers that cannot call cudaMalloc (device memory
owned by a pool or framework that grants no extra buffers, or a device footprint that
must not grow once running): same NLL as gf_nll, computed with the library's static
scratch array and no allocation.  Checked against gf_nll on two calls in a row, for a
grid-normalised tree (Voigtian + threshold) and an analytic one (exponential).

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
    # reference: the allocating path (gf_set_data + gf_nll)
    ref_ctx, ref_root, ref_obs = build()
    ref_ctx.set_data(ref_root, ref_obs, [x])
    # allocation-free path: a context holding only the model, caller-owned buffers
    ctx, root, obs = build()
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for th in thetas:  # two calls in a row, different theta
        ctx.nll_noalloc(root, obs, len(x), [xd.data_ptr()], th, out.data_ptr())
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
