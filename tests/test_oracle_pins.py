"""Pins of the CPU oracle against closed forms, library routines, invariants and
finite differences (no GPU).  Each test names the fact that fixes the expected value;
none of them re-types the oracle's own formula."""
from __future__ import annotations

import math

import mpmath
import numpy as np
import pytest
from scipy import integrate, optimize, special, stats

import oracle
from oracle import minimise
from paper_1311_1753_gb300 import synth
from tests import oracle_models as om

RNG = np.random.Generator(np.random.PCG64(4242))


# --------------------------------------------------------------------------------
# Faddeeva function (Voigtian, the paper's BW (x) Gaussian of Sec. 4 "Zach's fit")
# --------------------------------------------------------------------------------
def _w_mp(z):
    mpmath.mp.dps = 40
    zz = mpmath.mpc(z.real, z.imag)
    return complex(mpmath.exp(-zz * zz) * mpmath.erfc(-1j * zz))


def test_faddeeva_vs_mpmath_voigt_region():
    # The line-shape workload: y = Gamma/(2 sqrt2 sigma) ~ 0.094, Re z in [-14.2, 36.6]; widen both.
    x = RNG.uniform(-16, 40, 300)
    y = RNG.uniform(0.01, 0.3, 300)
    z = x + 1j * y
    w = oracle.faddeeva(z)
    ref = np.array([_w_mp(v) for v in z])
    assert np.max(np.abs(w - ref) / np.abs(ref)) < 1e-14
    # Re w (the Voigtian itself) relative to itself, not to |w|
    assert np.max(np.abs(w.real - ref.real) / np.abs(ref.real)) < 1e-12


def _trap_bound(z, w):
    # Rounding model of the pole-corrected trapezoid sum: the summand nearest the pole
    # is ~ h/(pi y) and cancels against the correction term, so the relative error is
    # a few ulps times (1 + h/(pi y |w|)), h = 0.4.
    return 8 * 2.2e-16 * (1 + 0.4 / (math.pi * z.imag * np.abs(w)))


def test_faddeeva_vs_mpmath_upper_half_plane():
    x = RNG.uniform(-8, 8, 300)
    y = 10 ** RNG.uniform(-3, 1.5, 300)
    z = x + 1j * y
    w = oracle.faddeeva(z)
    ref = np.array([_w_mp(v) for v in z])
    assert np.all(np.abs(w - ref) / np.abs(ref) < _trap_bound(z, ref))
    big = z.imag > 0.05
    assert np.max(np.abs(w - ref)[big] / np.abs(ref)[big]) < 1e-14


def test_faddeeva_imaginary_axis_is_erfcx():
    y = np.concatenate([10 ** np.linspace(-3, 2, 60)])
    w = oracle.faddeeva(1j * y)
    assert np.max(np.abs(w.imag)) < 1e-15
    ref = special.erfcx(y)
    assert np.all(np.abs(w.real / ref - 1) < _trap_bound(1j * y, ref))
    assert np.max(np.abs(w.real / ref - 1)[y > 0.05]) < 1e-14


def test_faddeeva_vs_scipy_wofz_grid():
    x, y = np.meshgrid(np.linspace(-30, 30, 121), np.array([0.02, 0.0943, 0.5, 3.0, 9.0]))
    z = (x + 1j * y).ravel()
    w = oracle.faddeeva(z)
    assert np.max(np.abs(w / special.wofz(z) - 1)) < 1e-13


def test_faddeeva_symmetry_and_asymptote():
    z = RNG.uniform(-10, 10, 50) + 1j * RNG.uniform(0.01, 5, 50)
    # w(-conj z) = conj w(z)
    assert np.max(np.abs(oracle.faddeeva(-np.conj(z)) - np.conj(oracle.faddeeva(z)))) < 1e-15
    # large |z|: w ~ i/(sqrt(pi) z) (1 + 1/(2 z^2) + 3/(4 z^4) + 15/(8 z^6))
    zl = np.array([35 + 0.1j, -33 + 0.05j, 31 + 2j, 40 + 0.0943j])
    asym = 1j / (math.sqrt(math.pi) * zl) * (1 + 1 / (2 * zl**2) + 3 / (4 * zl**4)
                                             + 15 / (8 * zl**6))
    assert np.max(np.abs(oracle.faddeeva(zl) / asym - 1)) < 1e-9


def test_faddeeva_real_axis_limit():
    # Re w(x + i0) = exp(-x^2); approach the axis (off the trapezoid nodes x = 0.4 n).
    x = np.array([0.13, 0.77, 1.51, 2.27, 3.03])
    w = oracle.faddeeva(x + 1e-9j)
    assert np.max(np.abs(w.real - np.exp(-x**2))) < 1e-8
    # Im w(x) = 2/sqrt(pi) Dawson(x)
    assert np.max(np.abs(w.imag - 2 / math.sqrt(math.pi) * special.dawsn(x))) < 1e-8


# --------------------------------------------------------------------------------
# Leaf PDFs and their normalisation
# --------------------------------------------------------------------------------
def _voigt_only(mu, s, w, lo, hi, nbins=10000):
    m = oracle.Model1D([(lo, hi)], nbins=nbins)
    v = m.voigt(0, m.param(mu), m.param(s), m.param(w))
    return m, v


def test_voigt_unit_integral_on_real_line():
    mu, s, w = 0.1455, 3e-4, 8e-5
    m, v = _voigt_only(mu, s, w, 0.0, 1.0)
    f = lambda x: m.leaf_shape(v, np.array([x]))[0]
    # Lorentzian tails: integrate in pieces around the peak, then add the analytic
    # Cauchy tail beyond +-L (Gaussian part is negligible there).
    L = 0.05
    core = sum(integrate.quad(f, a, b, epsabs=0, epsrel=1e-12, limit=400)[0]
               for a, b in [(mu - L, mu - 0.01), (mu - 0.01, mu), (mu, mu + 0.01),
                            (mu + 0.01, mu + L)])
    tail = 2 * (0.5 - math.atan(L / (w / 2)) / math.pi)
    assert abs(core + tail - 1) < 2e-7


def test_voigt_limits_lorentzian_and_gaussian():
    x = np.linspace(-0.01, 0.01, 41)
    # sigma -> 0: Cauchy with half-width Gamma/2
    m, v = _voigt_only(0.0, 1e-9, 1e-3, -1, 1)
    lor = stats.cauchy.pdf(x, 0.0, 0.5e-3)
    assert np.max(np.abs(m.leaf_shape(v, x) / lor - 1)) < 1e-8
    # Gamma -> 0: Gaussian
    m, v = _voigt_only(0.0, 3e-3, 1e-12, -1, 1)
    gau = stats.norm.pdf(x, 0.0, 3e-3)
    assert np.max(np.abs(m.leaf_shape(v, x) / gau - 1)) < 1e-8


def test_voigt_grid_norm_within_midpoint_bound():
    lo, hi = synth.VOIGT_RANGE
    mu, s, w = 0.1455, 3e-4, 8e-5
    m, v = _voigt_only(mu, s, w, lo, hi, nbins=10000)
    N, _ = m.norms()
    f = lambda x: m.leaf_shape(v, np.array([x]))[0]
    pts = [lo, mu - 0.003, mu - 0.0005, mu, mu + 0.0005, mu + 0.003, hi]
    exact = sum(integrate.quad(f, a, b, epsabs=0, epsrel=1e-13, limit=400)[0]
                for a, b in zip(pts[:-1], pts[1:]))
    h = (hi - lo) / 10000
    # |f''| is largest at the peak; bound it by a central difference there.
    e = 1e-6
    f2 = abs(f(mu + e) - 2 * f(mu) + f(mu - e)) / e**2
    bound = (hi - lo) * h**2 * f2 / 24
    assert abs(N[v] - exact) <= bound
    assert abs(N[v] / exact - 1) < 1e-5


def test_threshold_grid_norm_converges_to_incomplete_gamma():
    lo, hi = synth.VOIGT_RANGE
    c, p = 20.0, 0.5
    D = hi - lo
    exact = special.gammainc(p + 1, c * D) * special.gamma(p + 1) / c ** (p + 1)
    errs = []
    for nb in (1000, 10000, 100000):
        m = oracle.Model1D([(lo, hi)], nbins=nb)
        b = m.threshold(0, m.param(lo), m.param(p), m.param(c))
        N, _ = m.norms()
        errs.append(abs(N[b] - exact))
    # midpoint rule on a sqrt endpoint singularity: error ~ h^{3/2}
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 25 < r1 < 40 and 25 < r2 < 40
    assert errs[1] / exact < 1e-5


def test_exponential_norm_closed_form_and_truth_values():
    m, (a,) = om.exp_model(-1.0)
    N, dN = m.norms()
    # Int_0^10 e^{-x} dx = 1 - e^{-10}
    assert abs(N[0] - (1 - math.exp(-10))) < 1e-15
    assert abs(N[0] - 0.99995460) < 5e-9
    # E[x] = d log N / d alpha = Int x e^{-x} / N
    ex = integrate.quad(lambda x: x * math.exp(-x), 0, 10, epsabs=0, epsrel=1e-13)[0] / N[0]
    assert abs(dN[0, a] / N[0] - ex) < 1e-13
    assert abs(ex - 0.99954598) < 5e-9
    # near alpha = 0 (series branch) against quadrature
    for al in (1e-5, -3e-4, 0.0, 2.0, -7.5):
        m2, _ = om.exp_model(al)
        N2, dN2 = m2.norms()
        q = integrate.quad(lambda x: math.exp(al * x), 0, 10, epsabs=0, epsrel=1e-13)[0]
        qd = integrate.quad(lambda x: x * math.exp(al * x), 0, 10, epsabs=0, epsrel=1e-13)[0]
        assert abs(N2[0] / q - 1) < 1e-13 and abs(dN2[0, 0] / qd - 1) < 1e-12


def test_gaussian_norm_vs_normal_cdf():
    for mu, s, lo, hi in [(0.3, 0.2, -1, 1), (5.0, 0.5, -1, 1), (-3, 0.4, 0, 2)]:
        m = oracle.Model1D([(lo, hi)])
        g = m.gauss(0, m.param(mu), m.param(s))
        N, _ = m.norms()
        if mu > hi:  # both limits in the lower tail: difference of CDFs
            d = stats.norm.cdf(hi, mu, s) - stats.norm.cdf(lo, mu, s)
        else:
            d = stats.norm.sf(lo, mu, s) - stats.norm.sf(hi, mu, s)
        ref = s * math.sqrt(2 * math.pi) * d
        assert abs(N[g] / ref - 1) < 1e-12


def test_poly_norm_vs_quadrature():
    m = oracle.Model1D([(-1.0, 2.0)])
    co = [m.param(v) for v in (2.0, 0.3, -0.1, 0.05)]
    pn = m.poly(0, co)
    N, _ = m.norms()
    q = integrate.quad(lambda x: 2 + 0.3 * x - 0.1 * x**2 + 0.05 * x**3, -1, 2)[0]
    assert abs(N[pn] / q - 1) < 1e-14


# --------------------------------------------------------------------------------
# Combinators (Sec. 3): AddPdf fractions, ProdPdf separability
# --------------------------------------------------------------------------------
def test_add_pdf_integrates_to_one_on_grid():
    m, free = om.voigt_model(nbins=10000)
    lo, hi = synth.VOIGT_RANGE
    h = (hi - lo) / 10000
    xb = lo + (np.arange(10000) + 0.5) * h
    P = np.exp(m.logpdf([xb]))
    assert abs(h * P.sum() - 1) < 1e-12


def test_add_of_identical_children_ignores_fractions():
    lo, hi = 0.0, 3.0
    m = oracle.Model1D([(lo, hi)])
    mu, s = m.param(1.2), m.param(0.4)
    g1, g2, g3 = m.gauss(0, mu, s), m.gauss(0, mu, s), m.gauss(0, mu, s)
    f1, f2 = m.param(0.3), m.param(0.45)
    m.add([g1, g2, g3], [f1, f2])
    x = RNG.uniform(lo, hi, 100)
    single = oracle.Model1D([(lo, hi)])
    single.gauss(0, single.param(1.2), single.param(0.4))
    assert np.max(np.abs(m.logpdf([x]) - single.logpdf([x]))) < 1e-14


def test_add_three_components_vs_scipy_mixture():
    lo, hi = -2.0, 4.0
    m = oracle.Model1D([(lo, hi)])
    ga = m.gauss(0, m.param(0.5), m.param(0.3))
    ex = m.exp(0, m.param(-0.7))
    po = m.poly(0, [m.param(1.0), m.param(0.2)])
    m.add([ga, ex, po], [m.param(0.25), m.param(0.5)])
    x = RNG.uniform(lo, hi, 200)
    gpdf = stats.truncnorm.pdf(x, (lo - 0.5) / 0.3, (hi - 0.5) / 0.3, 0.5, 0.3)
    # truncated exponential and linear densities, normalised by scipy quadrature
    en = integrate.quad(lambda t: math.exp(-0.7 * t), lo, hi)[0]
    pn = integrate.quad(lambda t: 1 + 0.2 * t, lo, hi)[0]
    ref = 0.25 * gpdf + 0.5 * np.exp(-0.7 * x) / en + 0.25 * (1 + 0.2 * x) / pn
    assert np.max(np.abs(np.exp(m.logpdf([x])) / ref - 1)) < 1e-12


def test_prod_pdf_is_separable():
    # Listing 2: product of exponentials in x and y
    m = oracle.Model1D([(0.0, 5.0), (0.0, 5.0)])
    ex = m.exp(0, m.param(-2.4))
    ey = m.exp(1, m.param(-1.1))
    m.prod([ex, ey])
    x = synth.exp_events(1000, -2.4, 0, 5, seed=1)
    y = synth.exp_events(1000, -1.1, 0, 5, seed=2)
    mx = oracle.Model1D([(0.0, 5.0)]); mx.exp(0, mx.param(-2.4))
    my = oracle.Model1D([(0.0, 5.0)]); my.exp(0, my.param(-1.1))
    assert abs(m.nll([x, y]) - (mx.nll([x]) + my.nll([y]))) < 1e-10


# --------------------------------------------------------------------------------
# Gradients against central finite differences
# --------------------------------------------------------------------------------
def _fd_check(fun, p, idx, rel=1e-6):
    f0, g = fun(p)
    for k in idx:
        h = 1e-6 * max(1e-3, abs(p[k])) if abs(p[k]) > 0 else 1e-7
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (fun(pp)[0] - fun(pm)[0]) / (2 * h)
        scale = max(abs(g[k]), 1e-6 * abs(f0) / max(abs(p[k]), 1e-12))
        assert abs(fd - g[k]) <= rel * scale + 1e-7, (k, fd, g[k])


def test_gradient_exponential_fd():
    m, free = om.exp_model(-1.3)
    x = synth.exp_events(5000, -1.0)
    _fd_check(lambda p: m.nll([x], p, grad=True), m.p, free)


def test_gradient_voigt_fd():
    m, free = om.voigt_model(nbins=2000)
    lo, hi = synth.VOIGT_RANGE
    x = synth.voigt_threshold_events(3000, **synth.VOIGT_TRUTH, lo=lo, hi=hi)
    p = m.p
    p[free] *= np.array([1.00001, 1.02, 0.97, 1.05, 0.9])
    _fd_check(lambda q: m.nll([x], q, grad=True), p, free + [4], rel=2e-6)
    # x0 (fixed in the workload, free in general): the shape has a sqrt(x - x0) kink, so
    # difference away from it -- events and grid midpoints stay > 1e-4 above x0.
    m2, _ = om.voigt_model(nbins=2000)
    xx = x[x > lo + 1e-3]
    p2 = m2.p
    p2[3] = lo - 1e-4
    _fd_check(lambda q: m2.nll([xx], q, grad=True), p2, [3], rel=2e-6)


def test_gradient_gauss_poly_prod_fd():
    m = oracle.Model1D([(-1.0, 2.0), (0.0, 3.0)])
    g = m.gauss(0, m.param(0.4), m.param(0.6))
    po = m.poly(0, [m.param(1.0), m.param(0.3), m.param(0.1)])
    a = m.add([g, po], [m.param(0.6)])
    e = m.exp(1, m.param(-0.8))
    m.prod([a, e])
    x = RNG.uniform(-1, 2, 500)
    y = RNG.uniform(0, 3, 500)
    _fd_check(lambda q: m.nll([x, y], q, grad=True), m.p, list(range(len(m.values))))


# --------------------------------------------------------------------------------
# Dalitz kinematics and amplitudes (Sec. 4)
# --------------------------------------------------------------------------------
SPEC = om.load_dalitz_spec()
KIN = SPEC["kin"]


def _fourvectors(s12, s13):
    """Daughter four-momenta in the parent rest frame from (s12, s13): particle 3 along
    +z, particles 1 and 2 in the x-z plane (explicit construction, no invariant
    bounds).  Returns None outside the physical region."""
    M, m1, m2, m3 = KIN["M"], KIN["m1"], KIN["m2"], KIN["m3"]
    s23 = M**2 + m1**2 + m2**2 + m3**2 - s12 - s13
    E1 = (M**2 + m1**2 - s23) / (2 * M)
    E2 = (M**2 + m2**2 - s13) / (2 * M)
    E3 = (M**2 + m3**2 - s12) / (2 * M)
    if min(E1 - m1, E2 - m2, E3 - m3) < 0:
        return None
    p1, p2, p3 = (math.sqrt(E**2 - m**2) for E, m in ((E1, m1), (E2, m2), (E3, m3)))
    # p1 + p2 = -p3 (along -z); angle of p1 from law of cosines
    c1 = (p2**2 - p1**2 - p3**2) / (2 * p1 * p3)
    if abs(c1) > 1:
        return None
    s1 = math.sqrt(1 - c1 * c1)
    P1 = np.array([E1, p1 * s1, 0.0, p1 * c1])
    P3 = np.array([E3, 0.0, 0.0, p3])
    P2 = np.array([M, 0, 0, 0]) - P1 - P3
    return P1, P2, P3


def _mdot(a, b):
    return a[0] * b[0] - a[1:] @ b[1:]


def _boost_to_rest(p, frame):
    """Lorentz-boost four-vector p into the rest frame of four-vector ``frame``."""
    m = math.sqrt(_mdot(frame, frame))
    beta = frame[1:] / frame[0]
    b2 = beta @ beta
    g = frame[0] / m
    bp = beta @ p[1:]
    E = g * (p[0] - bp)
    vec = p[1:] + ((g - 1) * bp / b2 - g * p[0]) * beta if b2 > 0 else p[1:]
    return np.concatenate([[E], vec])


def test_dalitz_region_matches_explicit_kinematics():
    d = om.dalitz_from_spec(SPEC)
    x0, x1, y0, y1 = d.box()
    s12 = RNG.uniform(x0, x1, 4000)
    s13 = RNG.uniform(y0, y1, 4000)
    ins = d.inside(s12, s13)
    phys = np.array([_fourvectors(a, b) is not None for a, b in zip(s12, s13)])
    assert np.array_equal(ins, phys)
    # the constructed vectors reproduce the invariants (sum rule included)
    for a, b in zip(s12[ins][:50], s13[ins][:50]):
        P1, P2, P3 = _fourvectors(a, b)
        assert abs(_mdot(P1 + P2, P1 + P2) - a) < 1e-12
        assert abs(_mdot(P1 + P3, P1 + P3) - b) < 1e-12


def test_dalitz_area_converges_to_phase_space_integral():
    M, m1, m2, m3 = KIN["M"], KIN["m1"], KIN["m2"], KIN["m3"]

    def lam(a, b, c):
        return a * a + b * b + c * c - 2 * a * b - 2 * a * c - 2 * b * c

    # s13 range at fixed s12 from the Kallen function (textbook form, PDG kinematics)
    def width(s12):
        l1 = lam(s12, m1**2, m2**2)
        l2 = lam(M**2, s12, m3**2)
        return math.sqrt(max(l1, 0) * max(l2, 0)) / s12

    area = integrate.quad(width, (m1 + m2) ** 2, (M - m3) ** 2, epsabs=0, epsrel=1e-12,
                          limit=200)[0]
    d = om.dalitz_from_spec(SPEC)
    _, cnt = d.norm(anr=1.0 + 0j)
    x0, x1, y0, y1 = d.box()
    cell = (x1 - x0) * (y1 - y0) / (512 * 512)
    assert cnt == 155812
    assert abs(cnt * cell / area - 1) < 2e-3
    assert abs(area - 5.02525) < 2e-3
    # finer grids converge
    d2 = om.dalitz_from_spec(SPEC, 2048, 2048)
    _, cnt2 = d2.norm(anr=1.0 + 0j)
    assert abs(cnt2 * cell / 16 / area - 1) < abs(cnt * cell / area - 1)


def test_zemach_factors_vs_four_vectors():
    d = om.dalitz_from_spec(SPEC)
    x0, x1, y0, y1 = d.box()
    n = 0
    while n < 40:
        a, b = RNG.uniform(x0, x1), RNG.uniform(y0, y1)
        fv = _fourvectors(a, b)
        if fv is None:
            continue
        n += 1
        P = dict(zip((1, 2, 3), fv))
        for ch, (ia, ib, ic) in enumerate([(1, 2, 3), (1, 3, 2), (2, 3, 1)]):
            frame = P[ia] + P[ib]
            qa = _boost_to_rest(P[ia], frame)[1:]
            kc = _boost_to_rest(P[ic], frame)[1:]
            kq = kc @ qa
            k2, q2 = kc @ kc, qa @ qa
            s1 = d.zemach(ch, 1, a, b)
            s2 = d.zemach(ch, 2, a, b)
            assert abs(s1 - 4 * kq) < 1e-10 * max(1, abs(s1))
            assert abs(s2 - 16 * (kq * kq - k2 * q2 / 3)) < 1e-9 * max(1, abs(s2))


def test_breit_wigner_at_pole():
    d = om.dalitz_from_spec(SPEC)
    # place a point with s12 = m0^2 for each channel-0 resonance: A_r / S_L = i/(m0 G0)
    for r, res in enumerate(SPEC["resonances"]):
        if res["channel"] != 0:
            continue
        s12 = res["m0"] ** 2
        x0, x1, y0, y1 = d.box()
        grid = np.linspace(y0, y1, 2001)
        ins = d.inside(np.full_like(grid, s12), grid)
        s13 = grid[ins][len(grid[ins]) // 3]
        a = d.amp(r, np.array([s12]), np.array([s13]))[0]
        S = d.zemach(0, res["spin"], s12, s13)
        target = 1j / (res["m0"] * res["g0"])
        assert abs(a / S - target) < 1e-12 * abs(target)


def _barrier_hankel(L, x):
    """Blatt-Weisskopf barrier polynomial from the outgoing spherical wave:
    B_L = x^{2L} |x h_L(x)|^2 with h_L = j_L + i y_L (scipy's spherical Bessel
    functions), x = qR.  It is 1, 1 + x^2, 9 + 3x^2 + x^4 for L = 0, 1, 2 (von Hippel &
    Quigg 1972), here obtained without writing the polynomials."""
    h = special.spherical_jn(L, x) + 1j * special.spherical_yn(L, x)
    return x ** (2 * L) * np.abs(x * h) ** 2


def _two_body_q(m, ma, mb):
    """Momentum of a in the rest frame of mass m decaying to a, b (explicit energies)."""
    e = (m * m + ma * ma - mb * mb) / (2 * m)
    return math.sqrt(e * e - ma * ma)


@pytest.mark.parametrize("ch", [0, 1, 2])
@pytest.mark.parametrize("L", [0, 1, 2])
def test_breit_wigner_off_the_pole_vs_four_vectors(ch, L):
    """A_r = F_L S_L BW off the pole, for every channel and spin, against an independent
    construction: the pair's mass, the break-up momentum q and the bachelor momentum k
    from explicit four-vectors boosted into the pair's rest frame; q0 from the two-body
    energies at m0; the barrier factors from spherical Hankel functions; the running
    width Gamma(m) = Gamma0 (q/q0)^{2L+1} (m0/m) B_L(z0)/B_L(z); S_L from k and q.  A
    dropped power of q/q0 or a changed barrier polynomial moves A by far more than the
    tolerance at these points (|m - m0| up to ~1 GeV)."""
    k = SPEC["kin"]
    R = k["R"]
    names = [(1, 2, 3), (1, 3, 2), (2, 3, 1)]
    ia, ib, ic = names[ch]
    masses = {1: k["m1"], 2: k["m2"], 3: k["m3"]}
    ma, mb = masses[ia], masses[ib]
    rng = np.random.Generator(np.random.PCG64(900 + 10 * ch + L))
    for m0, g0 in ((0.77, 0.15), (1.27, 0.185), (0.98, 0.05)):
        d = oracle.Dalitz(k["M"], k["m1"], k["m2"], k["m3"], R)
        d.resonance(ch, L, d.param(m0), d.param(g0), d.param(1.0), d.param(0.0))
        x0, x1, y0, y1 = d.box()
        n = 0
        while n < 60:
            s12, s13 = rng.uniform(x0, x1), rng.uniform(y0, y1)
            fv = _fourvectors(s12, s13)
            if fv is None:
                continue
            n += 1
            P = dict(zip((1, 2, 3), fv))
            frame = P[ia] + P[ib]
            m = math.sqrt(_mdot(frame, frame))
            qa = _boost_to_rest(P[ia], frame)[1:]
            kc = _boost_to_rest(P[ic], frame)[1:]
            q = math.sqrt(qa @ qa)
            q0 = _two_body_q(m0, ma, mb)
            B, B0 = _barrier_hankel(L, q * R), _barrier_hankel(L, q0 * R)
            gam = g0 * (q / q0) ** (2 * L + 1) * (m0 / m) * B0 / B
            bw = 1.0 / (m0 * m0 - m * m - 1j * m0 * gam)
            kq, kk, qq = kc @ qa, kc @ kc, qa @ qa
            S = (1.0, 4 * kq, 16 * (kq * kq - kk * qq / 3))[L]
            Smax = (1.0, 4 * math.sqrt(kk * qq), 16 * kk * qq)[L]
            F = math.sqrt(B0 / B)
            want = F * S * bw
            got = d.amp(0, np.array([s12]), np.array([s13]))[0]
            assert abs(got - want) <= 1e-10 * F * Smax * abs(bw), (m0, s12, s13, got, want)


def test_dalitz_only_nonresonant_gives_log_area():
    d = om.dalitz_from_spec(SPEC)
    p = d.p.copy()
    p[2::4] = 0.0
    p[3::4] = 0.0
    s12 = np.array([0.5, 1.0, 1.3]); s13 = np.array([1.0, 0.9, 1.2])
    assert d.inside(s12, s13).all()
    N, cnt = d.norm(p)
    x0, x1, y0, y1 = d.box()
    area = cnt * (x1 - x0) * (y1 - y0) / 512**2
    assert abs(d.nll(s12, s13, p) - 3 * math.log(area)) < 1e-12


def test_dalitz_nll_invariant_under_common_rescaling():
    d = om.dalitz_from_spec(SPEC, 128, 128)
    s12, s13 = _inside_points(d, 300)
    p = d.p.copy()
    base = d.nll(s12, s13, p, anr=1.0 + 0j)
    lam = 0.7 * np.exp(0.9j)
    q = p.copy()
    c = (p[2::4] + 1j * p[3::4]) * lam
    q[2::4], q[3::4] = c.real, c.imag
    assert abs(d.nll(s12, s13, q, anr=lam) - base) < 1e-10 * abs(base)


def _inside_points(d, n, seed=7):
    rng = np.random.Generator(np.random.PCG64(seed))
    x0, x1, y0, y1 = d.box()
    s12, s13 = rng.uniform(x0, x1, 4 * n), rng.uniform(y0, y1, 4 * n)
    ins = d.inside(s12, s13)
    return s12[ins][:n].copy(), s13[ins][:n].copy()


def test_dalitz_gradient_fd():
    d = om.dalitz_from_spec(SPEC, 96, 96)
    s12, s13 = _inside_points(d, 200)
    p = d.p.copy()
    p[2::4] *= 1.05
    p[1::4] *= 0.97
    _fd_check(lambda q: d.nll(s12, s13, q, grad=True), p, list(range(len(p))), rel=1e-6)


def test_dalitz_amplitude_derivatives_fd():
    d = om.dalitz_from_spec(SPEC)
    s12, s13 = _inside_points(d, 50)
    for r, res in enumerate(SPEC["resonances"]):
        a, dm, dg = d.amp(r, s12, s13, deriv=True)
        for k, dd in ((4 * r, dm), (4 * r + 1, dg)):
            h = 1e-7
            pp, pm = d.p.copy(), d.p.copy()
            pp[k] += h
            pm[k] -= h
            fd = (d.amp(r, s12, s13, pp) - d.amp(r, s12, s13, pm)) / (2 * h)
            assert np.max(np.abs(fd - dd) / (np.abs(dd) + 1e-3 * np.abs(a))) < 1e-6


def test_dalitz_fit_fractions_sum_without_interference():
    # With resonances in distinct, non-overlapping... instead: the intensity integral is
    # a Hermitian form c^H G c; check N(c) = sum_rs conj(c_r) G_rs c_s with G assembled
    # from single and pairwise norms (polarisation identity).
    d = om.dalitz_from_spec(SPEC, 64, 64)
    p = d.p.copy()
    R = len(SPEC["resonances"])
    def N_of(cvec, anr):
        q = p.copy()
        q[2::4], q[3::4] = cvec.real, cvec.imag
        return d.norm(q, anr=anr)[0]
    G = np.zeros((R + 1, R + 1), complex)
    basis = lambda i: (np.eye(R)[i - 1] if i > 0 else np.zeros(R)).astype(complex)
    for i in range(R + 1):
        for j in range(R + 1):
            ci, cj = basis(i), basis(j)
            ai, aj = (1.0 if i == 0 else 0.0), (1.0 if j == 0 else 0.0)
            re = N_of(ci + cj, ai + aj) - N_of(ci - cj, ai - aj)
            im = N_of(ci + 1j * cj, ai + 1j * aj) - N_of(ci - 1j * cj, ai - 1j * aj)
            G[i, j] = (re - 1j * im) / 4
    c = np.concatenate([[1.0], p[2::4] + 1j * p[3::4]])
    assert np.allclose(G, G.conj().T, atol=1e-9)
    assert abs((c.conj() @ G @ c).real / d.norm(p)[0] - 1) < 1e-12


# --------------------------------------------------------------------------------
# Minimiser
# --------------------------------------------------------------------------------
def test_minimiser_quadratic_bowl():
    A = np.array([[4.0, 1.0, 0.5], [1.0, 3.0, 0.2], [0.5, 0.2, 2.0]])
    x_star = np.array([0.3, -1.2, 2.0])
    fg = lambda x: (0.5 * (x - x_star) @ A @ (x - x_star), A @ (x - x_star))
    r = minimise.fit(fg, np.zeros(3), step=np.full(3, 0.5), tol=1e-16)
    assert r.converged
    assert np.max(np.abs(r.x - x_star)) < 1e-8
    # f = NLL-like with up = 0.5: covariance = H^-1
    assert np.max(np.abs(r.cov - np.linalg.inv(A))) < 1e-8


def test_minimiser_rosenbrock_with_bounds():
    def fg(x):
        a, b = x
        f = (1 - a) ** 2 + 100 * (b - a * a) ** 2
        return f, np.array([-2 * (1 - a) - 400 * a * (b - a * a), 200 * (b - a * a)])
    r = minimise.fit(fg, np.array([-1.2, 1.0]), step=np.array([0.1, 0.1]),
                     lo=np.array([-5.0, -5.0]), hi=np.array([5.0, 5.0]), tol=1e-14)
    assert r.converged and np.max(np.abs(r.x - 1)) < 1e-5


def test_exponential_fit_matches_mle_root_and_error():
    m, (a,) = om.exp_model(-2.0)
    x = synth.exp_events(100_000, -1.0)
    mean = x.mean()

    # stationarity: mean(x) = E_alpha[x] = Int x e^{a x} / Int e^{a x} (quadrature)
    def ex(al):
        num = integrate.quad(lambda t: t * math.exp(al * t), 0, 10, epsabs=0, epsrel=1e-13)[0]
        den = integrate.quad(lambda t: math.exp(al * t), 0, 10, epsabs=0, epsrel=1e-13)[0]
        return num / den - mean

    root = optimize.brentq(ex, -1.5, -0.5, xtol=1e-15, rtol=1e-15)
    fg = lambda q: m.nll([x], np.array([q[0]]), grad=True)
    r = minimise.fit(fg, np.array([-2.0]), step=np.array([0.1]), lo=np.array([-10.0]),
                     hi=np.array([10.0]))
    assert r.converged
    # sigma_alpha = 1/sqrt(n Var_alpha(x)), Var from quadrature
    def var(al):
        den = integrate.quad(lambda t: math.exp(al * t), 0, 10)[0]
        m1 = integrate.quad(lambda t: t * math.exp(al * t), 0, 10)[0] / den
        m2 = integrate.quad(lambda t: t * t * math.exp(al * t), 0, 10)[0] / den
        return m2 - m1 * m1
    sig = 1 / math.sqrt(len(x) * var(root))
    assert abs(r.x[0] - root) < 1e-3 * sig
    assert abs(r.err[0] / sig - 1) < 1e-3
    assert abs(sig - 0.003169) < 2e-5


# --------------------------------------------------------------------------------
# Binned metrics (Sec. 2: the metric is separate from the PDF's evaluation; Sec. 4:
# the binned D*+ line-width fit)
# --------------------------------------------------------------------------------
def _exp_hist(alpha_true=-1.0, nb=40, lo=0.0, hi=10.0, n=20_000, seed=7):
    x = synth.exp_events(n, alpha_true, lo, hi, seed=seed)
    counts, edges = np.histogram(x, bins=nb, range=(lo, hi))
    return 0.5 * (edges[1:] + edges[:-1]), counts.astype(float), (hi - lo) / nb


def test_binned_multinomial_equals_unbinned_on_repeated_centres():
    """-sum n_b log P(x_b) is the unbinned NLL of a data set holding each centre n_b
    times (integer contents), value and gradient."""
    m, free = om.exp_model(-0.8)
    c, n, h = _exp_hist()
    rep = np.repeat(c, n.astype(int))
    fb, gb = m.binned([c], n, n.sum() * h, 0, grad=True)
    fu, gu = m.nll([rep], grad=True)
    assert abs(fb - fu) <= 1e-12 * abs(fu)
    assert abs(gb[0] - gu[0]) <= 1e-11 * abs(gu[0])


def test_binned_poisson_vs_scipy_logpmf():
    """Poisson metric = -sum log Poisson(n_b; nu_b) - sum log n_b! with nu_b from the
    closed-form truncated exponential density (scipy's pmf, no oracle density)."""
    alpha = -0.8
    m, free = om.exp_model(alpha)
    c, n, h = _exp_hist()
    K = n.sum() * h
    nu = K * alpha * np.exp(alpha * c) / np.expm1(alpha * 10.0)
    ref = -(stats.poisson.logpmf(n, nu) + special.gammaln(n + 1)).sum()
    assert abs(m.binned([c], n, K, 1) - ref) <= 1e-11 * abs(ref)


def test_binned_chisq_minimum_matches_curve_fit():
    """The chi-squared fit of a truncated Gaussian histogram (oracle metric + oracle BFGS)
    lands where scipy's least-squares curve_fit puts it, with its covariance."""
    lo, hi, nb = -3.0, 4.0, 70
    rng = np.random.Generator(np.random.PCG64(99))
    x = rng.normal(0.3, 0.8, 60_000)
    x = x[(x >= lo) & (x <= hi)]
    counts, edges = np.histogram(x, nb, (lo, hi))
    c = 0.5 * (edges[1:] + edges[:-1])
    h = (hi - lo) / nb
    n = counts.astype(float)
    s2 = np.maximum(n, 1.0)
    K = n.sum() * h

    def shape(xc, mu, s):
        return K * stats.truncnorm.pdf(xc, (lo - mu) / s, (hi - mu) / s, loc=mu, scale=s)

    popt, pcov = optimize.curve_fit(shape, c, n, p0=[0.2, 0.9], sigma=np.sqrt(s2),
                                    absolute_sigma=True)
    m = oracle.Model1D([(lo, hi)])
    m.gauss(0, m.param(0.2), m.param(0.9))
    r = minimise.fit(lambda q: m.binned([c], n, K, 2, s2=s2, p=q, grad=True),
                     np.array([0.2, 0.9]), step=np.array([0.05, 0.05]), up=1.0, tol=1e-12)
    assert r.converged
    err = np.sqrt(np.diag(pcov))
    assert np.all(np.abs(r.x - popt) <= 1e-4 * err), (r.x, popt)
    # curve_fit's covariance is the Gauss-Newton (J^T W J)^-1: equal to 2 H^-1 up to the
    # residual terms of the chi-squared Hessian (a few per cent here)
    assert np.all(np.abs(np.sqrt(np.diag(r.cov)) / err - 1) < 0.05)


@pytest.mark.parametrize("metric", [0, 1, 2])
def test_binned_metrics_gradient_fd(metric):
    m, free = om.voigt_model(nbins=2000)
    lo, hi = synth.VOIGT_RANGE
    x = synth.voigt_threshold_events(50_000, **synth.VOIGT_TRUTH, lo=lo, hi=hi)
    counts, edges = np.histogram(x, 500, (lo, hi))
    c = 0.5 * (edges[1:] + edges[:-1])
    n = counts.astype(float)
    K = n.sum() * (hi - lo) / 500
    p = m.p
    p[free] *= np.array([1.00001, 1.02, 0.97, 1.05, 0.9])
    _fd_check(lambda q: m.binned([c], n, K, metric, s2=np.maximum(n, 1.0), p=q, grad=True),
              p, free, rel=2e-6)


def test_binned_asimov_contents_are_stationary():
    """Contents equal to their expectation (n_b = nu_b(theta0)) make the Poisson and
    chi-squared metrics stationary at theta0, with chi-squared = 0 there."""
    m, free = om.voigt_model(nbins=400)
    lo, hi = synth.VOIGT_RANGE
    h = (hi - lo) / 400
    c = lo + (np.arange(400) + 0.5) * h
    K = 1e6 * h
    n = K * np.exp(m.logpdf([c]))
    q = m.p.copy()
    q[free] *= 1.001
    for metric in (1, 2):
        s2 = np.maximum(n, 1.0)
        f, g = m.binned([c], n, K, metric, s2=s2, grad=True)
        # scale: the same gradient 0.1 % away from theta0, parameter by parameter
        g1 = m.binned([c], n, K, metric, s2=s2, p=q, grad=True)[1]
        assert np.all(np.abs(g[free]) <= 1e-9 * np.abs(g1[free])), (metric, g[free], g1[free])
        if metric == 2:
            assert f <= 1e-18 * K


# --------------------------------------------------------------------------------
# ConvolutionPdf (Sec. 3) and the relativistic Breit-Wigner (Sec. 4, the D*+ fit)
# --------------------------------------------------------------------------------
D0_MASS, PI_MASS = 1.86484, 0.13957


def _lattice(lo, hi, L):
    return lo + np.arange(L + 1) * (hi - lo) / L


def test_conv_gauss_gauss_is_gauss_on_the_lattice():
    """Gaussian (mu, s1) convolved with a Gaussian resolution (0, s2) is a Gaussian of
    sigma sqrt(s1^2 + s2^2) (closed form); the lattice values of the normalised
    convolution match the truncated normal up to the interpolant's normalisation."""
    lo, hi, L = -4.0, 6.0, 2000
    s1, s2, mu = 0.7, 0.25, 0.9
    # a 10 sigma resolution window: at 8 sigma its cut tails already shift lattice values
    # 8 sigma_tot from mu by ~5e-10
    m = oracle.Model1D([(lo, hi), (-10 * s2, 10 * s2)])
    g1 = m.gauss(0, m.param(mu), m.param(s1))
    r = m.gauss(1, m.param(0.0), m.param(s2))
    m.conv(0, g1, r, L)
    xs = _lattice(lo, hi, L)
    P = np.exp(m.logpdf([xs]))
    st = math.hypot(s1, s2)
    ref = stats.truncnorm.pdf(xs, (lo - mu) / st, (hi - mu) / st, loc=mu, scale=st)
    # the trapezoid normalisation of the lattice values differs from the exact integral
    # by O(h^2 f''): compare shapes through the ratio, and the ratio to 1 within h^2
    ratio = P / ref
    assert np.max(np.abs(ratio / ratio.mean() - 1)) < 1e-10
    assert abs(ratio.mean() - 1) < ((hi - lo) / L) ** 2


def test_conv_interpolation_error_within_bound():
    """Between lattice points the value is the linear interpolant: its error against the
    closed form stays below h^2/8 max|f''|."""
    lo, hi, L = -4.0, 6.0, 400
    s1, s2, mu = 0.7, 0.25, 0.9
    m = oracle.Model1D([(lo, hi), (-8 * s2, 8 * s2)])
    m.conv(0, m.gauss(0, m.param(mu), m.param(s1)), m.gauss(1, m.param(0.0), m.param(s2)), L)
    h = (hi - lo) / L
    xs = lo + (np.arange(L) + 0.37) * h
    st = math.hypot(s1, s2)
    f = stats.truncnorm.pdf(xs, (lo - mu) / st, (hi - mu) / st, loc=mu, scale=st)
    fpp = np.max(np.abs(stats.norm.pdf(0) / st ** 3)) * 1.0  # max |f''| of the Gaussian
    err = np.abs(np.exp(m.logpdf([xs])) - f)
    assert np.max(err) <= h * h / 8 * fpp * 1.2 + 3 * h * h * np.max(f)


def test_conv_one_sided_exponential_is_exponnorm():
    """A one-sided exponential (threshold shape with power 0) convolved with a Gaussian
    is scipy's exponentially modified normal; the step of the model sits midway between
    model lattice points, so the Riemann sum errs by O(h^2)."""
    lo, hi, L = -1.0, 5.0, 3000
    h = (hi - lo) / L
    x0 = lo + 250.5 * h
    c, s = 1.3, 0.2
    m = oracle.Model1D([(lo, hi), (-9 * s, 9 * s)])
    th = m.threshold(0, m.param(x0), m.param(0.0), m.param(c))
    m.conv(0, th, m.gauss(1, m.param(0.0), m.param(s)), L)
    xs = _lattice(lo, hi, L)
    P = np.exp(m.logpdf([xs]))
    ref = stats.exponnorm.pdf(xs - x0, 1.0 / (c * s), scale=s)
    ref /= integrate.trapezoid(ref, xs)
    assert np.max(np.abs(P - ref)) < 2e-5 * np.max(ref)


def test_conv_voigt_gauss_is_voigt_profile():
    """Voigtian (sigma1, Gamma) convolved with a Gaussian (sigma2) is scipy's Voigt profile
    with sigma = sqrt(sigma1^2 + sigma2^2) (shapes compared on the lattice)."""
    lo, hi, L = 0.1395, 0.1610, 2150
    mu, s1, G, s2 = 0.1455, 2e-4, 8e-5, 2.5e-4
    m = oracle.Model1D([(lo, hi), (-10 * s2, 10 * s2)], nbins=20000)
    v = m.voigt(0, m.param(mu), m.param(s1), m.param(G))
    m.conv(0, v, m.gauss(1, m.param(0.0), m.param(s2)), L)
    xs = _lattice(lo, hi, L)
    P = np.exp(m.logpdf([xs]))
    ref = special.voigt_profile(xs - mu, math.hypot(s1, s2), G / 2)
    k = np.argmax(ref)
    # the Voigtian model is normalised on [lo, hi] (its Lorentzian tails reach outside):
    # compare shapes
    assert np.max(np.abs(P / P[k] - ref / ref[k])) < 2e-6


def test_conv_gradient_fd():
    lo, hi = 0.1395, 0.1610
    m = oracle.Model1D([(lo, hi), (-0.002, 0.002)], nbins=4000)
    v = m.voigt(0, m.param(0.1455), m.param(2e-4), m.param(8e-5))
    r1 = m.gauss(1, m.param(0.0), m.param(3e-4))
    r2 = m.gauss(1, m.param(1e-4), m.param(8e-4))
    res = m.add([r1, r2], [m.param(0.7)])
    m.conv(0, v, res, 860)
    x = synth.voigt_threshold_events(3000, **synth.VOIGT_TRUTH, lo=lo, hi=hi)
    p = m.p
    _fd_check(lambda q: m.nll([x], q, grad=True), p, list(range(8)), rel=2e-6)


def _relbw_model(lo, hi, dm0, g0, L=1, nbins=20000):
    m = oracle.Model1D([(lo, hi)], nbins=nbins)
    m.relbw(0, m.param(dm0), m.param(g0), m.param(D0_MASS), m.param(D0_MASS), m.param(PI_MASS),
            m.param(1.5), L)
    return m


def test_relbw_value_at_the_pole_and_threshold():
    """At m = m0 the running width equals Gamma0 and the shape is 1/(m0 Gamma0); at the
    D0 pi+ threshold it vanishes."""
    dm0, g0 = 0.14543, 8.3e-5
    m = _relbw_model(0.139, 0.16, dm0, g0)
    v = m.leaf_shape(0, np.array([dm0, PI_MASS + 1e-12, PI_MASS - 1e-6]))
    assert abs(v[0] * (dm0 + D0_MASS) * g0 - 1) < 1e-13
    assert v[1] < 1e-6 * v[0] and v[2] == 0.0


@pytest.mark.parametrize("L", [0, 1, 2])
def test_relbw_running_width_vs_two_body_momentum(L):
    """Gamma(m)/Gamma0 from the shape (f D/m) against (q/q0)^{2L+1} (m0/m) B_L(z0)/B_L(z)
    with q the pion momentum computed from explicit two-body energies and the barrier
    polynomials from spherical Hankel functions."""
    dm0, g0 = 0.14543, 8.3e-5
    m = _relbw_model(0.139, 0.16, dm0, g0, L=L)
    xs = np.array([0.1420, 0.1450, 0.1500, 0.1580])
    f = m.leaf_shape(0, xs)
    M, M0 = xs + D0_MASS, dm0 + D0_MASS

    def q(mm):
        e = (mm * mm + PI_MASS ** 2 - D0_MASS ** 2) / (2 * mm)
        return np.sqrt(e * e - PI_MASS ** 2)
    B = _barrier_hankel(L, q(M) * 1.5)
    B0 = _barrier_hankel(L, q(M0) * 1.5)
    G = g0 * (q(M) / q(M0)) ** (2 * L + 1) * (M0 / M) * B0 / B
    D = (M0 ** 2 - M ** 2) ** 2 + M0 ** 2 * G ** 2
    assert np.max(np.abs(f * D / (M * G) - 1)) < 1e-12


def test_relbw_narrow_limit_is_cauchy():
    """For Gamma0 -> 0 the normalised line shape near the pole approaches a Cauchy
    density of half-width Gamma0/2 in m; at an offset d from the pole the P-wave factor
    (q/q0)^3 ~ (1 + d/(dm0 - threshold))^(3/2) tilts it by ~ 1.5 d/(dm0 - threshold)."""
    dm0, g0 = 0.1455, 2e-6
    lo, hi = dm0 - 2e-4, dm0 + 2e-4
    m = _relbw_model(lo, hi, dm0, g0, nbins=100000)
    xs = np.linspace(dm0 - 2e-5, dm0 + 2e-5, 41)
    P = np.exp(m.logpdf([xs]))
    ref = stats.cauchy.pdf(xs, dm0, g0 / 2)
    ref /= stats.cauchy.cdf(hi, dm0, g0 / 2) - stats.cauchy.cdf(lo, dm0, g0 / 2)
    tilt = 1.5 * np.abs(xs - dm0) / (dm0 - PI_MASS)
    assert np.all(np.abs(P / ref - 1) <= 1.2 * tilt + 2e-4)


def test_relbw_gradient_fd():
    lo, hi = 0.1395, 0.1610
    m = _relbw_model(lo, hi, 0.14543, 8.3e-5, nbins=4000)
    x = synth.voigt_threshold_events(3000, **synth.VOIGT_TRUTH, lo=lo, hi=hi)
    p = m.p
    f0, g = m.nll([x], p, grad=True)
    # steps well below the width 8.3e-5 (the curvature scale of the line shape)
    for k, h in ((0, 3e-9), (1, 1e-11)):
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (m.nll([x], pp) - m.nll([x], pm)) / (2 * h)
        assert abs(fd / g[k] - 1) < 1e-7, (k, fd, g[k])


# --------------------------------------------------------------------------------
# MappedPdf and CompositePdf (Sec. 3)
# --------------------------------------------------------------------------------
def test_mapped_two_gaussians_piecewise_closed_form():
    """Child k on its interval, each child normalised on the whole range: against the
    truncated normal densities of scipy, normalised by the exact piecewise integral (the
    boundary on a grid edge: the midpoint rule then errs by O(h^2) only)."""
    lo, hi, nb = -2.0, 4.0, 6000
    b = lo + 2500 * (hi - lo) / nb
    m = oracle.Model1D([(lo, hi)], nbins=nb)
    g1 = m.gauss(0, m.param(0.3), m.param(0.5))
    g2 = m.gauss(0, m.param(1.8), m.param(1.1))
    m.mapped(0, [g1, g2], [m.param(b)])
    xs = np.linspace(lo, hi, 997)
    P = np.exp(m.logpdf([xs]))
    t1 = stats.truncnorm((lo - 0.3) / 0.5, (hi - 0.3) / 0.5, loc=0.3, scale=0.5)
    t2 = stats.truncnorm((lo - 1.8) / 1.1, (hi - 1.8) / 1.1, loc=1.8, scale=1.1)
    Z = (t1.cdf(b) - t1.cdf(lo)) + (t2.cdf(hi) - t2.cdf(b))
    ref = np.where(xs < b, t1.pdf(xs), t2.pdf(xs)) / Z
    h = (hi - lo) / nb
    assert np.max(np.abs(P / ref - 1)) < 4 * h * h


def test_mapped_identical_children_is_the_child():
    lo, hi = 0.0, 10.0
    m = oracle.Model1D([(lo, hi)], nbins=20000)
    a = m.param(-0.4)
    e1, e2, e3 = m.exp(0, a), m.exp(0, a), m.exp(0, a)
    m.mapped(0, [e1, e2, e3], [m.param(3.0), m.param(7.5)])
    xs = np.linspace(lo, hi, 301)
    ref = -0.4 * np.exp(-0.4 * xs) / np.expm1(-0.4 * 10.0)
    assert np.max(np.abs(np.exp(m.logpdf([xs])) / ref - 1)) < ((hi - lo) / 20000) ** 2


def test_composite_exp_of_linear_is_exponential():
    """exp(a g(x)) with the linear core g = c0 + c1 x is the exponential of rate a c1."""
    lo, hi, nb = 0.0, 5.0, 10000
    m = oracle.Model1D([(lo, hi), (-50.0, 50.0)], nbins=nb)
    core = m.poly(0, [m.param(0.7), m.param(1.3)])
    shell = m.exp(1, m.param(-0.45))
    m.composite(0, core, shell)
    xs = np.linspace(lo, hi, 211)
    rate = -0.45 * 1.3
    ref = rate * np.exp(rate * xs) / np.expm1(rate * hi)
    # the second observable only carries the shell's range: one data column
    P = np.exp(oracle_logpdf_1col(m, xs))
    assert np.max(np.abs(P / ref - 1)) < 2 * ((hi - lo) / nb) ** 2


def test_composite_gauss_of_linear_is_gauss():
    """A Gaussian shell (mu, s) of the core c0 + c1 x is a Gaussian in x of mean
    (mu - c0)/c1 and width s/|c1| (scipy's truncated normal)."""
    lo, hi, nb = -3.0, 3.0, 12000
    c0, c1, mu, s = 0.4, -1.7, 0.9, 1.2
    m = oracle.Model1D([(lo, hi), (-50.0, 50.0)], nbins=nb)
    m.composite(0, m.poly(0, [m.param(c0), m.param(c1)]), m.gauss(1, m.param(mu), m.param(s)))
    xs = np.linspace(lo, hi, 301)
    mx, sx = (mu - c0) / c1, s / abs(c1)
    ref = stats.truncnorm.pdf(xs, (lo - mx) / sx, (hi - mx) / sx, loc=mx, scale=sx)
    P = np.exp(oracle_logpdf_1col(m, xs))
    assert np.max(np.abs(P / ref - 1)) < 2 * ((hi - lo) / nb) ** 2 * 4


def oracle_logpdf_1col(m, xs):
    return m.logpdf([xs])


@pytest.mark.parametrize("which", ["mapped", "composite"])
def test_mapped_composite_gradient_fd(which):
    x = synth.exp_events(2000, -0.5, 0.0, 5.0, seed=9)
    if which == "mapped":
        m = oracle.Model1D([(0.0, 5.0)], nbins=4000)
        g = m.gauss(0, m.param(1.0), m.param(0.8))
        e = m.exp(0, m.param(-0.6))
        po = m.poly(0, [m.param(1.0), m.param(0.3)])
        m.mapped(0, [g, e, po], [m.param(1.7), m.param(3.2)])
        idx = [0, 1, 2, 4]
    else:
        m = oracle.Model1D([(0.0, 5.0), (-50.0, 50.0)], nbins=4000)
        m.composite(0, m.poly(0, [m.param(0.2), m.param(0.9), m.param(-0.05)]),
                    m.gauss(1, m.param(1.0), m.param(1.5)))
        idx = [0, 1, 2, 3, 4]
    _fd_check(lambda q: m.nll([x], q, grad=True), m.p, idx, rel=2e-6)


# --------------------------------------------------------------------------------
# Time-dependent Dalitz model (Sec. 4: the D0 -> pi+ pi- pi0 mixing fit)
# --------------------------------------------------------------------------------
@pytest.mark.parametrize("lam", [2.4, 2.4 * (1 - 0.3j), 2.4 * (1 + 0.05j)])
@pytest.mark.parametrize("sig", [0.05, 0.3])
def test_smeared_exponential_vs_quadrature(lam, sig):
    """Int_0^inf e^{-lam u} Gauss(t - u; sigma) du by adaptive quadrature."""
    ts = np.array([-0.8, -0.1, 0.0, 0.2, 1.0, 3.5])
    T = oracle.smeared_exp(complex(lam), ts, sig)
    for t, v in zip(ts, T):
        f = lambda u, part: (np.exp(-complex(lam) * u) * stats.norm.pdf(t - u, scale=sig)).__getattribute__(part)
        ref = (integrate.quad(f, 0, np.inf, args=("real",), epsabs=0, epsrel=1e-13, limit=200)[0]
               + 1j * integrate.quad(f, 0, np.inf, args=("imag",), epsabs=0, epsrel=1e-13, limit=200)[0])
        assert abs(v - ref) <= 1e-11 * max(abs(ref), 1e-3), (t, v, ref)


def test_smeared_exponential_real_rate_is_exponnorm():
    lam, sig = 2.4, 0.12
    ts = np.linspace(-1.0, 6.0, 57)
    T = oracle.smeared_exp(lam, ts, sig).real
    ref = stats.exponnorm.pdf(ts, 1.0 / (lam * sig), scale=sig) / lam
    assert np.max(np.abs(T / ref - 1)) < 1e-12


def _tddp_model(nbx=48, nby=48, tau=0.41, x=0.01, y=0.007, scale=1.1):
    spec = om.load_dalitz_spec()
    k = spec["kin"]
    d = oracle.Tddp(k["M"], k["m1"], k["m2"], k["m3"], k["R"], nbx, nby)
    for r in spec["resonances"]:
        idx = [d.param(r[f]) for f in ("m0", "g0", "re", "im")]
        d.resonance(r["channel"], r["spin"], *idx)
    d.time_params(d.param(tau), d.param(x), d.param(y), d.param(scale))
    return d, spec


def _tddp_events(d, spec, n, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    s12, s13 = synth.dalitz_events(n, om.dalitz_accept(d, spec["envelope"]), seed=seed)
    sigt = rng.uniform(0.05, 0.15, n)
    t = rng.exponential(0.41, n) + sigt * rng.standard_normal(n)
    return s12, s13, t, sigt


def test_tddp_without_mixing_is_dalitz_times_exponnorm():
    """x = y = 0: the intensity factorises into |A|^2 and the smeared exponential, so
    the NLL is the (separately pinned) Dalitz NLL plus -sum log of scipy's exponentially
    modified normal density."""
    d, spec = _tddp_model(x=0.0, y=0.0)
    s12, s13, t, sigt = _tddp_events(d, spec, 300)
    f = d.nll_t(s12, s13, t, sigt)
    dz = om.dalitz_from_spec(spec, nbx=48, nby=48)
    fd = dz.nll(s12, s13)
    tau, sc = 0.41, 1.1
    ft = -np.sum(np.log(stats.exponnorm.pdf(t, tau / (sc * sigt), scale=sc * sigt)))
    assert abs(f - (fd + ft)) <= 1e-11 * abs(f)


def test_tddp_time_integral_of_the_intensity():
    """Integrating the smeared intensity over t reproduces the time integral of the
    unsmeared mixing formula (quadrature of e^{-Gt} cosh/cos/sinh/sin)."""
    d, spec = _tddp_model()
    tau, x, y = 0.41, 0.01, 0.007
    G = 1 / tau
    for s12, s13 in ((0.9, 1.1), (1.6, 0.7), (0.4, 2.1)):
        assert d.inside([s12], [s13])[0]
        A = 1 + sum((r["re"] + 1j * r["im"]) * d.amp(i, [s12], [s13])[0]
                    for i, r in enumerate(spec["resonances"]))
        s23 = sum(v ** 2 for v in (spec["kin"]["M"], spec["kin"]["m1"], spec["kin"]["m2"],
                                   spec["kin"]["m3"])) - s12 - s13
        B = 1 + sum((r["re"] + 1j * r["im"]) * d.amp(i, [s12], [s23])[0]
                    for i, r in enumerate(spec["resonances"]))
        aa, bb, xab = abs(A) ** 2, abs(B) ** 2, np.conj(A) * B

        def unsmeared(u):
            e = math.exp(-G * u)
            return e * (0.5 * (aa + bb) * math.cosh(y * G * u) + 0.5 * (aa - bb) * math.cos(x * G * u)
                        + xab.real * math.sinh(y * G * u) - xab.imag * math.sin(x * G * u))
        ref = integrate.quad(unsmeared, 0, np.inf, epsabs=0, epsrel=1e-12, limit=200)[0]
        got = integrate.quad(lambda u: d.intensity_t([s12], [s13], [u], [0.1])[0], -2.0, 12.0,
                             points=[0.0], epsabs=0, epsrel=1e-12, limit=400)[0]
        assert abs(got / ref - 1) < 1e-9


def test_tddp_gradient_fd():
    d, spec = _tddp_model(nbx=24, nby=24)
    s12, s13, t, sigt = _tddp_events(d, spec, 200)
    p = d.p
    free = [i for i in range(len(p)) if i % 4 >= 2 and i < 32] + [32, 33, 34, 35]
    _fd_check(lambda q: d.nll_t(s12, s13, t, sigt, p=q, grad=True), p, free, rel=2e-6)


def _tddp_dens_model(nbx=24, nby=24, b=(2.3, 0.4, -0.3), rng_=(0.02, 0.5)):
    d, spec = _tddp_model(nbx, nby)
    tp = d.tp
    d.time_params(tp.p_tau, tp.p_x, tp.p_y, tp.p_s,
                  density=tuple(d.param(v) for v in b), sigt_range=rng_)
    return d, spec


def test_sigt_density_integrates_to_one_at_every_dalitz_point():
    """The sigma_t density is normalised on its range at any (s12, s13) and parameters:
    adaptive quadrature of exp(log D) over [slo, shi]."""
    d, spec = _tddp_dens_model()
    lo, hi = 0.02, 0.5
    x0, x1, y0, y1 = d.box()
    for b in ((2.3, 0.4, -0.3), (0.5, -1.0, 2.0), (4.0, 0.0, 0.0)):
        p = d.p.copy()
        p[-3:] = b
        for s12, s13 in ((0.9, 1.1), (0.3, 2.5), (2.6, 0.2)):
            f = lambda st: math.exp(d.sigt_logd([s12], [s13], [st], p)[0])
            val = integrate.quad(f, lo, hi, epsabs=0, epsrel=1e-13, limit=200)[0]
            assert abs(val - 1) < 1e-11, (b, s12, s13, val)


def test_sigt_density_is_a_truncated_gamma():
    """At a point where the rate is exp(b0) (the plot's centre, or b1 = b2 = 0) the density
    is scipy's Gamma(2, scale 1/rate) renormalised on [slo, shi]."""
    lo, hi = 0.02, 0.5
    d, spec = _tddp_dens_model(b=(2.1, 0.0, 0.0), rng_=(lo, hi))
    lam = math.exp(2.1)
    st = np.linspace(lo, hi, 57)
    g = stats.gamma(2.0, scale=1.0 / lam)
    ref = g.pdf(st) / (g.cdf(hi) - g.cdf(lo))
    got = np.exp(d.sigt_logd(np.full_like(st, 1.0), np.full_like(st, 1.2), st))
    assert np.max(np.abs(got / ref - 1)) < 1e-12
    # and with slopes, at the centre of the plot
    k = spec["kin"]
    sc = (k["M"] ** 2 + k["m1"] ** 2 + k["m2"] ** 2 + k["m3"] ** 2) / 3
    p = d.p.copy()
    p[-2:] = (0.7, -0.4)
    got = np.exp(d.sigt_logd(np.full_like(st, sc), np.full_like(st, sc), st, p))
    assert np.max(np.abs(got / ref - 1)) < 1e-12


def test_tddp_shape_and_density_gradient_fd():
    """The mixing likelihood with free resonance masses and widths and the sigma_t density
    (38 parameters here): analytic gradient against central differences."""
    d, spec = _tddp_dens_model(nbx=20, nby=20)
    s12, s13, t, sigt = _tddp_events(d, spec, 150)
    sigt = np.clip(sigt, 0.021, 0.49)
    p = d.p
    _fd_check(lambda q: d.nll_t(s12, s13, t, sigt, p=q, grad=True), p, list(range(len(p))),
              rel=3e-6)


def test_tddp_norm_is_grid_sum_of_time_integrals():
    """N(theta) = sum over the inside cell centres of dA x the integral over all t of the
    intensity: per cell the integral of the unsmeared mixing formula over t >= 0 by
    quadrature (Gaussian smearing keeps the integral), with large x and y so that every
    mixing term (cosh, cos, sinh, sin with A and the CP-conjugate B) weighs in."""
    tau, x, y = 0.41, 0.2, 0.15
    d, spec = _tddp_model(nbx=10, nby=10, tau=tau, x=x, y=y)
    N = d.norm_t()
    x0, x1, y0, y1 = d.box()
    hx, hy = (x1 - x0) / 10, (y1 - y0) / 10
    k = spec["kin"]
    msum = k["M"] ** 2 + k["m1"] ** 2 + k["m2"] ** 2 + k["m3"] ** 2
    G = 1 / tau
    ref, ncell = 0.0, 0
    for i in range(10):
        for j in range(10):
            s12, s13 = x0 + (i + 0.5) * hx, y0 + (j + 0.5) * hy
            if not d.inside([s12], [s13])[0]:
                continue
            ncell += 1
            s23 = msum - s12 - s13
            A = 1 + sum((r["re"] + 1j * r["im"]) * d.amp(q, [s12], [s13])[0]
                        for q, r in enumerate(spec["resonances"]))
            B = 1 + sum((r["re"] + 1j * r["im"]) * d.amp(q, [s12], [s23])[0]
                        for q, r in enumerate(spec["resonances"]))
            aa, bb, xab = abs(A) ** 2, abs(B) ** 2, np.conj(A) * B

            def unsmeared(u):
                # e^{-Gu} cosh(yGu), e^{-Gu} sinh(yGu) as sums of decaying exponentials
                e1, e2, e = math.exp(-G * (1 - y) * u), math.exp(-G * (1 + y) * u), math.exp(-G * u)
                return (0.5 * (aa + bb) * 0.5 * (e1 + e2) + 0.5 * (aa - bb) * e * math.cos(x * G * u)
                        + xab.real * 0.5 * (e1 - e2) - xab.imag * e * math.sin(x * G * u))
            ref += hx * hy * integrate.quad(unsmeared, 0, np.inf, epsabs=0, epsrel=1e-13,
                                            limit=200)[0]
    assert ncell > 30
    assert abs(N / ref - 1) < 1e-10, (N, ref)


def test_oracle_pool_sums_match_the_single_process_oracle():
    """The full-size parity tests split the oracle's Dalitz sums over spawned worker
    processes: the slice sums equal the one-process sums (up to summation order) and the
    pooled accept-reject draws the same events."""
    from tests import oracle_pool as op
    d = om.dalitz_from_spec(SPEC, 64, 64)
    s12, s13 = _inside_points(d, 1001)
    p = d.p.copy()
    p[2::4] *= 1.02
    f1, g1 = d.nll(s12, s13, p, grad=True)
    f2, g2 = op.dalitz_nll(SPEC, p, s12, s13, 64, 64, grad=True)
    assert abs(f2 - f1) <= 1e-12 * abs(f1)
    assert np.allclose(g2, g1, rtol=1e-11, atol=1e-11 * np.abs(g1).max())
    P1, k1 = d.intensity(s12, s13, p, kappa=True)
    P2, k2 = op.dalitz_intensity(SPEC, p, s12, s13, kappa=True)
    assert np.array_equal(P1, P2) and np.array_equal(k1, k2)
    a = synth.dalitz_events(500, om.dalitz_accept(om.dalitz_from_spec(SPEC), SPEC["envelope"]), 5,
                            batch=4096)
    b = synth.dalitz_events(500, op.dalitz_accept(SPEC), 5, batch=4096)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
