"""Element-wise parity checks shared by the GPU tests.

The bar per event is 1e-12 relative on P: |P_gpu/P_orc - 1| <= 1e-12, i.e.
|log P_gpu - log P_orc| <= 1e-12 for every event (log P is compared directly; the two
differ by the relative error of P to first order).  Where the oracle supplies a
condition number kappa_i of the evaluation (the Dalitz interference number
(|a_NR| + sum |c_r A_r|)^2 / |A|^2), the bound is 1e-12 * max(1, kappa_i)."""
from __future__ import annotations

import numpy as np

WORST: dict[str, float] = {}


def per_event(name, lg, lo, kappa=None, tol=1e-12):
    """Assert |lg_i - lo_i| <= tol * max(1, kappa_i) for every i; record the worst ratio
    of error to bound (and the worst absolute error) under `name`."""
    lg = np.asarray(lg, dtype=float)
    lo = np.asarray(lo, dtype=float)
    assert lg.shape == lo.shape
    if lg.size == 0:
        return 0.0
    err = np.abs(lg - lo)
    bound = tol * (np.maximum(1.0, kappa) if kappa is not None else 1.0)
    ratio = err / bound
    k = int(np.argmax(ratio))
    WORST[name] = float(err.max())
    assert np.all(np.isfinite(lg)), name
    assert ratio[k] <= 1.0, (f"{name}: event {k}: |d log P| = {err[k]:.3e} > bound "
                             f"{np.broadcast_to(bound, err.shape)[k]:.3e} (log P = {lo[k]})")
    return float(err.max())
