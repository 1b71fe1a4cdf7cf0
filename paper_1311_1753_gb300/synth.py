"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 4).

This module draws random numbers and nothing else: it holds none of the likelihood
arithmetic.  Where a sample must follow a model density (the Dalitz toy data), the
caller supplies the accept/reject decision as a callable, so the same generator
serves the CUDA library (bench) and the CPU oracle (tests) without either importing
the other.

All generators use numpy ``Generator(PCG64(seed))``.
"""
from __future__ import annotations

import math

import numpy as np

# Workload seeds (the paper's datasets are private; these stand in for them).
SEED_EXP = 17531
SEED_VOIGT = 17532
SEED_DALITZ_MODEL = 17533
SEED_DALITZ_EVENTS = 17543
SEED_DALITZ_BIG = 17534
SEED_ARRIVALS = 17535

# D0 -> pi+ pi- pi0 kinematics (GeV): parent, pi+, pi-, pi0.
D0_MASS, PIC_MASS, PI0_MASS = 1.8648, 0.13957, 0.13498

# The 1D composite workload: a narrow peak on the D*+ - D0 mass-difference range with
# a threshold background (the unbinned analogue of the paper's D*+ line-width fit).
VOIGT_RANGE = (0.1395, 0.1610)
VOIGT_TRUTH = dict(mu=0.1455, sigma=3e-4, width=8e-5, x0=0.1395, power=0.5, c=20.0, frac=0.3)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def exp_events(n: int, alpha: float, lo: float = 0.0, hi: float = 10.0, seed: int = SEED_EXP):
    """n draws from e^{alpha x} on [lo, hi]: an exponential variate from the nearer edge
    (rate |alpha|), redrawn until it falls inside the range."""
    rng = _rng(seed)
    out = np.empty(0)
    while len(out) < n:
        m = int((n - len(out)) * 1.1) + 16
        if alpha == 0.0:
            x = rng.uniform(lo, hi, m)
        else:
            e = rng.standard_exponential(m) / abs(alpha)
            x = lo + e if alpha < 0 else hi - e
        x = x[(x >= lo) & (x <= hi)]
        out = np.concatenate([out, x])
    return out[:n].copy()


def voigt_threshold_events(n: int, mu: float, sigma: float, width: float, x0: float, power: float,
                           c: float, frac: float, lo: float, hi: float, seed: int = SEED_VOIGT):
    """n draws from frac * Voigt + (1 - frac) * threshold, each component truncated to
    [lo, hi].  The Voigtian is drawn as its defining convolution (a Gaussian variate of
    std sigma plus a Cauchy variate of half-width width/2); the threshold shape
    (x-x0)^power e^{-c(x-x0)} is a Gamma(power+1, 1/c) variate shifted by x0.  Draws
    outside the range are rejected and redrawn, component by component."""
    rng = _rng(seed)
    is_sig = rng.random(n) < frac
    nsig = int(is_sig.sum())

    def draw(k, one):
        got = np.empty(0)
        while len(got) < k:
            x = one(int((k - len(got)) * 1.3) + 16)
            got = np.concatenate([got, x[(x >= lo) & (x <= hi)]])
        return got[:k]

    sig = draw(nsig, lambda m: mu + sigma * rng.standard_normal(m)
               + 0.5 * width * rng.standard_cauchy(m))
    bkg = draw(n - nsig, lambda m: x0 + rng.gamma(power + 1.0, 1.0 / c, m))
    out = np.empty(n)
    out[is_sig] = sig
    out[~is_sig] = bkg
    return out


def dalitz_box(M=D0_MASS, m1=PIC_MASS, m2=PIC_MASS, m3=PI0_MASS):
    """Bounding box of the Dalitz plot in (m12^2, m13^2)."""
    return ((m1 + m2) ** 2, (M - m3) ** 2, (m1 + m3) ** 2, (M - m2) ** 2)


def dalitz_model_draw(seed: int = SEED_DALITZ_MODEL, nres: int = 8):
    """Seeded resonance list: mass in U(0.5, 1.7) GeV, width in U(0.05, 0.4) GeV, spin in
    U{0,1,2}, channel r mod 3, coefficient magnitude rho in U(0.5, 1.5) and phase in
    U(-pi, pi).  A draw whose mass lies within the sum of the widths of an earlier
    resonance with the same channel and spin is redrawn (two such resonances are nearly
    the same amplitude, which leaves their masses and widths without a unique fit).  The
    caller rescales the magnitudes by its own normalisation integrals."""
    rng = _rng(seed)
    res = []
    for r in range(nres):
        while True:
            m0 = rng.uniform(0.5, 1.7)
            g0 = rng.uniform(0.05, 0.4)
            spin = int(rng.integers(0, 3))
            clash = any(q["channel"] == r % 3 and q["spin"] == spin
                        and abs(q["m0"] - m0) < q["g0"] + g0 for q in res)
            if not clash:
                break
        rho = rng.uniform(0.5, 1.5)
        phi = rng.uniform(-math.pi, math.pi)
        res.append(dict(channel=r % 3, spin=spin, m0=m0, g0=g0, rho=rho, phi=phi))
    return res


def dalitz_events(n: int, accept, seed: int, box=None, batch: int = 1 << 20):
    """n points (s12, s13) by accept-reject: uniform candidates in the bounding box and a
    uniform variate u per candidate; ``accept(s12, s13, u) -> bool mask`` is the caller's
    decision (inside the region and u * envelope < density).  Accepted points keep
    their draw order."""
    rng = _rng(seed)
    x0, x1, y0, y1 = dalitz_box() if box is None else box
    xs, ys = [], []
    got = 0
    while got < n:
        s12 = rng.uniform(x0, x1, batch)
        s13 = rng.uniform(y0, y1, batch)
        u = rng.random(batch)
        m = np.asarray(accept(s12, s13, u), dtype=bool)
        xs.append(s12[m])
        ys.append(s13[m])
        got += int(m.sum())
    return np.concatenate(xs)[:n].copy(), np.concatenate(ys)[:n].copy()


def poisson_arrivals(nreq: int, rate: float, seed: int = SEED_ARRIVALS):
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = _rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, nreq))


def serving_requests(nreq: int = 256, nmin: int = 10_000, nmax: int = 4_000_000,
                     seed: int = SEED_ARRIVALS):
    """Per request: model kind (0 = 1D composite, 1 = Dalitz, by a fair coin), event count
    log-uniform in [nmin, nmax], and its own data seed 1,000,000 + j."""
    rng = _rng(seed + 1)
    kinds = (rng.random(nreq) < 0.5).astype(int)
    counts = np.exp(rng.uniform(math.log(nmin), math.log(nmax), nreq)).astype(np.int64)
    seeds = 1_000_000 + np.arange(nreq)
    return kinds, counts, seeds
