"""Plain quasi-Newton minimiser for the oracle (test infrastructure only).

The paper hands the NLL to MINUIT's Migrad (Sec. 2: FitManager calls DefineParameter
for every fit variable, then mnmigr), and notes that any search algorithm could take
its place.  This is a textbook BFGS (Nocedal & Wright, Numerical Optimization,
Alg. 6.1) with a strong-Wolfe line search (Alg. 3.5/3.6), on MINUIT's internal
coordinates for bounded parameters:

    ext = lo + (hi - lo) (sin(u) + 1) / 2

Convergence: estimated distance to minimum EDM = g^T V g / 2 below ``tol``, with V the
BFGS inverse-Hessian estimate.  Errors: the Hessian of the NLL in external coordinates
by central differences of the analytic gradient at the minimum; covariance =
2 up H^-1 (up = 0.5 for a negative log-likelihood).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class FitResult:
    x: np.ndarray
    err: np.ndarray
    cov: np.ndarray
    fval: float
    edm: float
    ncalls: int
    converged: bool
    history: list = field(default_factory=list)


class _Transform:
    def __init__(self, lo, hi):
        self.lo = np.asarray(lo, dtype=float)
        self.hi = np.asarray(hi, dtype=float)
        self.bounded = self.hi > self.lo

    def to_int(self, x):
        u = np.array(x, dtype=float)
        b = self.bounded
        r = 2 * (u[b] - self.lo[b]) / (self.hi[b] - self.lo[b]) - 1
        u[b] = np.arcsin(np.clip(r, -1, 1))
        return u

    def to_ext(self, u):
        x = np.array(u, dtype=float)
        b = self.bounded
        x[b] = self.lo[b] + (self.hi[b] - self.lo[b]) * (np.sin(u[b]) + 1) / 2
        return x

    def dext(self, u):
        d = np.ones_like(u)
        b = self.bounded
        d[b] = (self.hi[b] - self.lo[b]) * np.cos(u[b]) / 2
        return d


def _line_search(phi, f0, d0, a1=1.0, c1=1e-4, c2=0.9, maxit=40):
    """Strong-Wolfe step along a descent direction; phi(a) -> (f, dphi)."""

    def zoom(alo, ahi, flo, dlo):
        for _ in range(maxit):
            a = 0.5 * (alo + ahi)
            f, d = phi(a)
            if f > f0 + c1 * a * d0 or f >= flo:
                ahi = a
            else:
                if abs(d) <= -c2 * d0:
                    return a, f
                if d * (ahi - alo) >= 0:
                    ahi = alo
                alo, flo, dlo = a, f, d
        return (alo, flo) if flo < f0 else (None, None)

    a_prev, f_prev, d_prev = 0.0, f0, d0
    a = a1
    for i in range(maxit):
        f, d = phi(a)
        if not math.isfinite(f) or f > f0 + c1 * a * d0 or (i > 0 and f >= f_prev):
            if not math.isfinite(f):
                # shrink into the finite region first
                a = 0.5 * (a_prev + a)
                continue
            return zoom(a_prev, a, f_prev, d_prev)
        if abs(d) <= -c2 * d0:
            return a, f
        if d >= 0:
            return zoom(a, a_prev, f, d)
        a_prev, f_prev, d_prev = a, f, d
        a *= 2.0
    return (a_prev, f_prev) if f_prev < f0 else (None, None)


def fit(fg, x0, step, lo=None, hi=None, up=0.5, tol=1e-8, max_iter=1000) -> FitResult:
    """Minimise fg(x) -> (f, grad) from x0 with MINUIT-style bounds (lo < hi bounds
    the parameter; lo == hi leaves it free)."""
    n = len(x0)
    lo = np.zeros(n) if lo is None else np.asarray(lo, float)
    hi = np.zeros(n) if hi is None else np.asarray(hi, float)
    tr = _Transform(lo, hi)
    calls = [0]

    def fgi(u):
        calls[0] += 1
        x = tr.to_ext(u)
        f, g = fg(x)
        return f, np.asarray(g, float) * tr.dext(u)

    u = tr.to_int(np.asarray(x0, float))
    f, g = fgi(u)
    sint = np.asarray(step, float) / np.maximum(np.abs(tr.dext(u)), 1e-300)
    V = np.diag(sint ** 2)
    edm = 0.5 * g @ V @ g
    converged = False
    hist = []
    for it in range(max_iter):
        p = -V @ g
        d0 = g @ p
        if d0 >= 0:
            V = np.diag(sint ** 2)
            p = -V @ g
            d0 = g @ p

        cache = {}

        def phi(a):
            fa, ga = fgi(u + a * p)
            cache[a] = ga
            return fa, ga @ p

        a, fa = _line_search(phi, f, d0)
        if a is None:
            if edm < 10 * tol:
                converged = True
            break
        s = a * p
        u_new = u + s
        g_new = cache[a]
        y = g_new - g
        sy = s @ y
        if it == 0 and sy > 0:
            V = (sy / (y @ y)) * np.eye(n)
        if sy > 1e-300:
            rho = 1.0 / sy
            I = np.eye(n)
            V = (I - rho * np.outer(s, y)) @ V @ (I - rho * np.outer(y, s)) + rho * np.outer(s, s)
        u, f, g = u_new, fa, g_new
        edm = 0.5 * g @ V @ g
        hist.append((f, edm))
        if edm < tol:
            converged = True
            break

    x = tr.to_ext(u)
    # Hessian in external coordinates by central differences of the gradient.
    sig = np.sqrt(np.abs(np.diag(V))) * np.abs(tr.dext(u))
    h = np.where(sig > 0, 1e-2 * sig, 1e-6 * np.maximum(1, np.abs(x)))
    H = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = h[k]
        _, gp = fg(x + e)
        _, gm = fg(x - e)
        calls[0] += 2
        H[:, k] = (np.asarray(gp) - np.asarray(gm)) / (2 * h[k])
    H = 0.5 * (H + H.T)
    cov = 2 * up * np.linalg.inv(H)
    err = np.sqrt(np.abs(np.diag(cov)))
    return FitResult(x, err, cov, f, edm, calls[0], converged, hist)
