"""The oracle over the host cores, for the full-size parity tests (tests only).

A process pool started with `spawn` (safe after the parent process has initialised CUDA)
whose workers rebuild the oracle's Dalitz model from its plain description and evaluate
one contiguous slice of the events each.  Sums over slices add up to the oracle's sum
over all events (the n log N term is additive in n); only the order of the additions
differs."""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_POOL = None


def cores() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def pool():
    global _POOL
    if _POOL is None:
        _POOL = mp.get_context("spawn").Pool(min(16, cores()))
    return _POOL


def _slices(n, k):
    edges = np.linspace(0, n, k + 1).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


def _w_intensity(args):
    from tests import oracle_models as om
    spec, p, s12, s13, kappa = args
    d = om.dalitz_from_spec(spec)
    return d.intensity(s12, s13, p, kappa=kappa)


def _w_nll(args):
    from tests import oracle_models as om
    spec, nbx, nby, p, s12, s13, grad = args
    d = om.dalitz_from_spec(spec, nbx, nby)
    return d.nll(s12, s13, p, grad=grad)


def dalitz_intensity(spec, p, s12, s13, kappa=False):
    """|A|^2 (and the interference condition number) of every event."""
    parts = _slices(len(s12), 4 * min(16, cores()))
    res = pool().map(_w_intensity, [(spec, p, s12[a:b], s13[a:b], kappa) for a, b in parts])
    if kappa:
        return np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res])
    return np.concatenate(res)


def dalitz_nll(spec, p, s12, s13, nbx=512, nby=512, grad=False):
    """-sum log |A_i|^2 + n log N (and its gradient), summed over slices."""
    parts = _slices(len(s12), min(16, cores()))
    res = pool().map(_w_nll, [(spec, nbx, nby, p, s12[a:b], s13[a:b], grad) for a, b in parts])
    if grad:
        return sum(r[0] for r in res), np.sum([r[1] for r in res], axis=0)
    return sum(res)


def dalitz_accept(spec):
    """accept(s12, s13, u) for synth.dalitz_events with the oracle's density, over the pool."""
    from tests import oracle_models as om
    d = om.dalitz_from_spec(spec)
    env = spec["envelope"]
    p = d.p

    def acc(s12, s13, u):
        inside = d.inside(s12, s13)
        out = np.zeros(len(s12), dtype=bool)
        idx = np.nonzero(inside)[0]
        if len(idx):
            P = dalitz_intensity(spec, p, s12[idx], s13[idx])
            out[idx] = u[idx] * env < P
        return out
    return acc


def _w_tddp(args):
    from tests import oracle_models as om
    spec, nb, time, dens, p, cols, grad = args
    d = om.tddp_from_spec(spec, nb, time, dens)
    return d.nll_t(*cols, p=p, grad=grad)


def tddp_nll(spec, nb, time, dens, p, cols, grad=False):
    """The mixing model's NLL (and gradient) summed over slices of the events."""
    parts = _slices(len(cols[0]), min(16, cores()))
    res = pool().map(_w_tddp, [(spec, nb, time, dens, p, [c[a:b] for c in cols], grad)
                               for a, b in parts])
    if grad:
        return sum(r[0] for r in res), np.sum([r[1] for r in res], axis=0)
    return sum(res)
