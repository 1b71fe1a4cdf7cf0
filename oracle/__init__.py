"""FP64 CPU oracle for the unbinned NLL path of GooFit (arXiv:1311.1753).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline``/``--impl reference`` legs of ``bench.py`` may import this package.
The product library never loads it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C99, FP64, no FMA contraction); this
module compiles it with gcc on first use and wraps it with ctypes.  Model objects
mirror the paper's vocabulary (Sec. 2): observables with ranges, parameters, PDFs
combined by sums and products (Sec. 3), and a three-body Dalitz amplitude model
(Sec. 4).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

# Leaf and combinator codes, as in oracle.c.
EXP, GAUSS, VOIGT, THRESH, POLY, RELBW, ADD, PROD, CONV, MAPPED, COMPOSITE = (
    1, 2, 3, 4, 5, 6, 10, 11, 12, 13, 14)
MAXPAR, MAXCHILD = 16, 8


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liborc.so (gcc, -O2, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class OrcNode(C.Structure):
    _fields_ = [("type", C.c_int32), ("obs", C.c_int32), ("npar", C.c_int32),
                ("par", C.c_int32 * MAXPAR), ("nchild", C.c_int32), ("child", C.c_int32 * MAXCHILD),
                ("aux", C.c_int32)]


class OrcModel(C.Structure):
    _fields_ = [("nnodes", C.c_int32), ("root", C.c_int32), ("nodes", C.POINTER(OrcNode)),
                ("nobs", C.c_int32), ("lo", C.POINTER(C.c_double)), ("hi", C.POINTER(C.c_double)),
                ("nbins", C.c_int32), ("ndata", C.c_int32)]


class OrcDkin(C.Structure):
    _fields_ = [("M", C.c_double), ("m1", C.c_double), ("m2", C.c_double), ("m3", C.c_double),
                ("R", C.c_double)]


class OrcRes(C.Structure):
    _fields_ = [("channel", C.c_int32), ("spin", C.c_int32), ("p_m0", C.c_int32),
                ("p_g0", C.c_int32), ("p_re", C.c_int32), ("p_im", C.c_int32)]


_D = C.POINTER(C.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            so = C.CDLL(build())
            so.orc_faddeeva.argtypes = [C.c_double, C.c_double, _D, _D]
            so.orc_faddeeva_many.argtypes = [C.c_int64, _D, _D, _D, _D]
            so.orc_norms.argtypes = [C.POINTER(OrcModel), _D, C.c_int, _D, _D]
            so.orc_norms.restype = C.c_int
            so.orc_logpdf.argtypes = [C.POINTER(OrcModel), _D, C.c_int, C.c_int64, C.POINTER(_D), _D]
            so.orc_logpdf.restype = C.c_int
            so.orc_nll.argtypes = [C.POINTER(OrcModel), _D, C.c_int, C.c_int64, C.POINTER(_D), _D, _D]
            so.orc_nll.restype = C.c_int
            so.orc_binned.argtypes = [C.POINTER(OrcModel), _D, C.c_int, C.c_int64, C.POINTER(_D),
                                      _D, _D, C.c_double, C.c_int, _D, _D]
            so.orc_binned.restype = C.c_int
            so.orc_leaf_shape_many.argtypes = [C.POINTER(OrcNode), _D, C.c_int64, _D, _D]
            so.orc_dalitz_inside.argtypes = [C.POINTER(OrcDkin), C.c_double, C.c_double]
            so.orc_dalitz_inside_many.argtypes = [C.POINTER(OrcDkin), C.c_int64, _D, _D,
                                                  C.POINTER(C.c_int8)]
            so.orc_dalitz_amp_many.argtypes = [C.POINTER(OrcDkin), C.c_int, C.c_int, C.c_double,
                                               C.c_double, C.c_int64, _D, _D, _D, _D, _D]
            so.orc_dalitz_norm.argtypes = [C.POINTER(OrcDkin), C.c_int, C.POINTER(OrcRes), _D,
                                           C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, _D,
                                           _D, C.POINTER(C.c_int64)]
            so.orc_dalitz_intensity.argtypes = [C.POINTER(OrcDkin), C.c_int, C.POINTER(OrcRes), _D,
                                                C.c_int, C.c_double, C.c_double, C.c_int64, _D, _D,
                                                _D, _D]
            so.orc_dalitz_nll.argtypes = [C.POINTER(OrcDkin), C.c_int, C.POINTER(OrcRes), _D,
                                          C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                          C.c_int64, _D, _D, _D, _D]
            so.orc_zemach_at.argtypes = [C.POINTER(OrcDkin), C.c_int, C.c_int, C.c_double,
                                         C.c_double]
            so.orc_zemach_at.restype = C.c_double
            _lib = so
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def faddeeva(z) -> np.ndarray:
    """w(z) = exp(-z^2) erfc(-iz) for Im z > 0 (pole-corrected trapezoidal rule)."""
    z = np.asarray(z, dtype=np.complex128)
    flat = z.ravel()
    x, y = _f64(flat.real), _f64(flat.imag)
    re, im = np.empty_like(x), np.empty_like(x)
    lib().orc_faddeeva_many(len(x), _dp(x), _dp(y), _dp(re), _dp(im))
    return (re + 1j * im).reshape(z.shape)


class Model1D:
    """A PDF tree over one or more observables (Sec. 2-3 of the paper).

    Parameters are held in one flat array (fixed and free alike); nodes refer to
    them by index, like GooFit's index arrays (Listing 3-4)."""

    def __init__(self, obs_ranges, nbins: int = 10000):
        self.lo = _f64([r[0] for r in obs_ranges])
        self.hi = _f64([r[1] for r in obs_ranges])
        self.nbins = int(nbins)
        self._ndata = len(self.lo)
        self.values: list[float] = []
        self.nodes: list[OrcNode] = []
        self.root = -1

    # parameters -------------------------------------------------------------
    def param(self, value: float) -> int:
        self.values.append(float(value))
        return len(self.values) - 1

    @property
    def p(self) -> np.ndarray:
        return _f64(self.values)

    # nodes ---------------------------------------------------------------------
    def _node(self, typ, obs=0, pars=(), children=(), aux=0) -> int:
        nd = OrcNode()
        nd.type, nd.obs, nd.npar, nd.nchild, nd.aux = typ, obs, len(pars), len(children), aux
        assert len(pars) <= MAXPAR and len(children) <= MAXCHILD
        for i, q in enumerate(pars):
            nd.par[i] = q
        for i, c in enumerate(children):
            nd.child[i] = c
        self.nodes.append(nd)
        self.root = len(self.nodes) - 1
        return self.root

    def exp(self, obs, alpha):
        return self._node(EXP, obs, [alpha])

    def gauss(self, obs, mu, sigma):
        return self._node(GAUSS, obs, [mu, sigma])

    def voigt(self, obs, mu, sigma, width):
        return self._node(VOIGT, obs, [mu, sigma, width])

    def threshold(self, obs, x0, power, c):
        return self._node(THRESH, obs, [x0, power, c])

    def poly(self, obs, coefs):
        return self._node(POLY, obs, list(coefs))

    def relbw(self, obs, dm0, gamma0, shift, ma, mb, radius, spin=1):
        """Relativistic Breit-Wigner line shape in x = m - shift (Sec. 4's D*+ fit: a
        P-wave resonance in the D*+ - D0 mass difference)."""
        return self._node(RELBW, obs, [dm0, gamma0, shift, ma, mb, radius], aux=int(spin))

    def conv(self, obs, model, resolution, lattice):
        """ConvolutionPdf (Sec. 3): model (a node over obs) convolved with resolution (a
        node over its own residual observable, declared after the data observables) on a
        lattice of `lattice` bins of obs's range."""
        return self._node(CONV, obs, [], [model, resolution], aux=int(lattice))

    def mapped(self, obs, children, bounds):
        """MappedPdf (Sec. 3): child k on [b_{k-1}, b_k) of obs's range; bounds are the
        n-1 interior boundaries (parameter indices, normally fixed)."""
        assert len(bounds) == len(children) - 1
        return self._node(MAPPED, obs, list(bounds), list(children))

    def composite(self, obs, core, shell):
        """CompositePdf (Sec. 3): shell(core(x)), both unnormalised leaf shapes, the
        result normalised on obs's range (midpoint rule, nbins)."""
        return self._node(COMPOSITE, obs, [], [core, shell])

    def add(self, children, fracs):
        assert len(fracs) == len(children) - 1
        return self._node(ADD, 0, list(fracs), list(children))

    def prod(self, children):
        return self._node(PROD, 0, [], list(children))

    # evaluation -------------------------------------------------------------------
    def _model(self):
        arr = (OrcNode * len(self.nodes))(*self.nodes)
        m = OrcModel(len(self.nodes), self.root, arr, len(self.lo), _dp(self.lo), _dp(self.hi),
                     self.nbins, self._ndata)
        return m, arr

    def _cols(self, cols):
        cols = [_f64(c) for c in cols]
        # one auxiliary observable per convolution (its residual variable) and per
        # composite (its shell's argument), declared after the data observables
        nres = sum(1 for nd in self.nodes if nd.type in (CONV, COMPOSITE))
        if len(cols) != len(self.lo) - nres or any(len(c) != len(cols[0]) for c in cols):
            raise ValueError(f"the model has {len(self.lo) - nres} data observables: one "
                             "column each, all of the same length")
        self._ndata = len(cols)
        ptrs = (_D * len(cols))(*[_dp(c) for c in cols])
        return cols, ptrs

    def norms(self, p=None):
        p = self.p if p is None else _f64(p)
        m, keep = self._model()
        N = np.empty(len(self.nodes))
        dN = np.empty(len(self.nodes) * len(p))
        rc = lib().orc_norms(C.byref(m), _dp(p), len(p), _dp(N), _dp(dN))
        assert rc == 0
        return N, dN.reshape(len(self.nodes), len(p))

    def logpdf(self, cols, p=None) -> np.ndarray:
        p = self.p if p is None else _f64(p)
        cols, ptrs = self._cols(cols)
        m, keep = self._model()
        out = np.empty(len(cols[0]))
        rc = lib().orc_logpdf(C.byref(m), _dp(p), len(p), len(out), ptrs, _dp(out))
        assert rc == 0
        return out

    def nll(self, cols, p=None, grad: bool = False):
        p = self.p if p is None else _f64(p)
        cols, ptrs = self._cols(cols)
        m, keep = self._model()
        out = np.zeros(1)
        g = np.zeros(len(p)) if grad else None
        rc = lib().orc_nll(C.byref(m), _dp(p), len(p), len(cols[0]), ptrs, _dp(out),
                           _dp(g) if grad else None)
        assert rc == 0
        return (out[0], g) if grad else out[0]

    def binned(self, centres, counts, K, metric, s2=None, p=None, grad: bool = False):
        """Binned metric over bins with the given centres (one column per observable) and
        contents: 0 multinomial -sum n log P, 1 Poisson sum nu - n log nu, 2 chi-squared
        sum (n - nu)^2/s2, with nu = K P(centre)."""
        p = self.p if p is None else _f64(p)
        cols, ptrs = self._cols(centres)
        m, keep = self._model()
        n = _f64(counts)
        assert len(n) == len(cols[0])
        v = _f64(s2) if s2 is not None else None
        out = np.zeros(1)
        g = np.zeros(len(p)) if grad else None
        rc = lib().orc_binned(C.byref(m), _dp(p), len(p), len(n), ptrs, _dp(n),
                              _dp(v) if v is not None else None, float(K), int(metric),
                              _dp(out), _dp(g) if grad else None)
        assert rc == 0
        return (out[0], g) if grad else out[0]

    def leaf_shape(self, node: int, x, p=None) -> np.ndarray:
        p = self.p if p is None else _f64(p)
        x = _f64(x)
        out = np.empty_like(x)
        lib().orc_leaf_shape_many(C.byref(self.nodes[node]), _dp(p), len(x), _dp(x), _dp(out))
        return out


class Dalitz:
    """Three-body Dalitz amplitude model on (s12, s13) (Sec. 4 of the paper).

    A = a_NR + sum_r c_r F_L S_L BW_r;  P = |A|^2 normalised on an nbx x nby
    cell-centre grid over the kinematic region."""

    def __init__(self, M, m1, m2, m3, R=1.5, nbx=512, nby=512):
        self.kin = OrcDkin(M, m1, m2, m3, R)
        self.nbx, self.nby = int(nbx), int(nby)
        self.values: list[float] = []
        self.res: list[OrcRes] = []

    def param(self, value: float) -> int:
        self.values.append(float(value))
        return len(self.values) - 1

    @property
    def p(self) -> np.ndarray:
        return _f64(self.values)

    def resonance(self, channel, spin, m0, g0, re, im) -> int:
        self.res.append(OrcRes(channel, spin, m0, g0, re, im))
        return len(self.res) - 1

    def box(self):
        k = self.kin
        return ((k.m1 + k.m2) ** 2, (k.M - k.m3) ** 2, (k.m1 + k.m3) ** 2, (k.M - k.m2) ** 2)

    def _resarr(self):
        return (OrcRes * max(1, len(self.res)))(*self.res)

    def inside(self, s12, s13) -> np.ndarray:
        s12, s13 = _f64(s12), _f64(s13)
        out = np.empty(len(s12), dtype=np.int8)
        lib().orc_dalitz_inside_many(C.byref(self.kin), len(s12), _dp(s12), _dp(s13),
                                     out.ctypes.data_as(C.POINTER(C.c_int8)))
        return out.astype(bool)

    def amp(self, r: int, s12, s13, p=None, deriv: bool = False):
        p = self.p if p is None else _f64(p)
        rs = self.res[r]
        s12, s13 = _f64(s12), _f64(s13)
        re, im = np.empty_like(s12), np.empty_like(s12)
        d = np.empty(4 * len(s12)) if deriv else None
        lib().orc_dalitz_amp_many(C.byref(self.kin), rs.channel, rs.spin, p[rs.p_m0], p[rs.p_g0],
                                  len(s12), _dp(s12), _dp(s13), _dp(re), _dp(im),
                                  _dp(d) if deriv else None)
        a = re + 1j * im
        if deriv:
            d = d.reshape(-1, 4)
            return a, d[:, 0] + 1j * d[:, 1], d[:, 2] + 1j * d[:, 3]
        return a

    def zemach(self, channel: int, spin: int, s12: float, s13: float) -> float:
        return lib().orc_zemach_at(C.byref(self.kin), channel, spin, s12, s13)

    def norm(self, p=None, anr=1.0 + 0j, grad=False):
        p = self.p if p is None else _f64(p)
        N = np.zeros(1)
        dN = np.zeros(len(p)) if grad else None
        cnt = C.c_int64(0)
        lib().orc_dalitz_norm(C.byref(self.kin), len(self.res), self._resarr(), _dp(p), len(p),
                              anr.real, anr.imag, self.nbx, self.nby, _dp(N),
                              _dp(dN) if grad else None, C.byref(cnt))
        return (N[0], dN, cnt.value) if grad else (N[0], cnt.value)

    def intensity(self, s12, s13, p=None, anr=1.0 + 0j, kappa=False):
        p = self.p if p is None else _f64(p)
        s12, s13 = _f64(s12), _f64(s13)
        P = np.empty_like(s12)
        K = np.empty_like(s12) if kappa else None
        lib().orc_dalitz_intensity(C.byref(self.kin), len(self.res), self._resarr(), _dp(p), len(p),
                                   anr.real, anr.imag, len(s12), _dp(s12), _dp(s13), _dp(P),
                                   _dp(K) if kappa else None)
        return (P, K) if kappa else P

    def nll(self, s12, s13, p=None, anr=1.0 + 0j, grad=False):
        p = self.p if p is None else _f64(p)
        s12, s13 = _f64(s12), _f64(s13)
        out = np.zeros(1)
        g = np.zeros(len(p)) if grad else None
        lib().orc_dalitz_nll(C.byref(self.kin), len(self.res), self._resarr(), _dp(p), len(p),
                             anr.real, anr.imag, self.nbx, self.nby, len(s12), _dp(s12), _dp(s13),
                             _dp(out), _dp(g) if grad else None)
        return (out[0], g) if grad else out[0]


class OrcTpar(C.Structure):
    _fields_ = [("p_tau", C.c_int32), ("p_x", C.c_int32), ("p_y", C.c_int32), ("p_s", C.c_int32),
                ("dens", C.c_int32), ("p_b0", C.c_int32), ("p_b1", C.c_int32),
                ("p_b2", C.c_int32), ("slo", C.c_double), ("shi", C.c_double)]


def _tddp_lib():
    so = lib()
    if not getattr(so, "_tddp_ready", False):
        so.orc_smeared_exp_many.argtypes = [C.c_int64, C.c_double, C.c_double, _D, C.c_double,
                                            _D, _D]
        args = [C.POINTER(OrcDkin), C.c_int, C.POINTER(OrcRes), C.POINTER(OrcTpar), _D, C.c_int]
        so.orc_tddp_intensity.argtypes = args + [C.c_int64, _D, _D, _D, _D, _D]
        so.orc_tddp_norm.argtypes = args + [C.c_int, C.c_int, _D]
        so.orc_tddp_norm.restype = C.c_double
        so.orc_tddp_nll.argtypes = args + [C.c_int, C.c_int, C.c_int64, _D, _D, _D, _D, _D, _D]
        so.orc_sigt_logd_many.argtypes = [C.POINTER(OrcDkin), C.POINTER(OrcTpar), _D, C.c_int64,
                                          _D, _D, _D, _D, _D]
        so._tddp_ready = True
    return so


def smeared_exp(lam: complex, t, sigma: float) -> np.ndarray:
    """Int_0^inf e^{-lam u} Gauss(t - u; sigma) du (complex lam, Re lam > 0)."""
    t = _f64(t)
    re, im = np.empty_like(t), np.empty_like(t)
    _tddp_lib().orc_smeared_exp_many(len(t), lam.real, lam.imag, _dp(t), float(sigma), _dp(re),
                                      _dp(im))
    return re + 1j * im


class Tddp(Dalitz):
    """Time-dependent Dalitz model (Sec. 4: the D0 mixing fit): the Dalitz amplitude model
    for D0 (A) and D0bar (B, at the point with particles 1 and 2 exchanged), decay time
    with mixing (tau, x, y) convolved with a Gaussian of width scale * sigma_t."""

    def __init__(self, M, m1, m2, m3, R=1.5, nbx=512, nby=512):
        super().__init__(M, m1, m2, m3, R, nbx, nby)
        self.tp = None

    def time_params(self, tau, x, y, scale, density=None, sigt_range=(0.0, 1.0)):
        """density: (b0, b1, b2) parameter indices of the sigma_t density (a Gamma(2)
        distribution on sigt_range with rate exp(b0 + b1 (s12 - sc) + b2 (s13 - sc))),
        or None for the likelihood conditional on sigma_t."""
        if density is None:
            self.tp = OrcTpar(tau, x, y, scale, 0, 0, 0, 0, *sigt_range)
        else:
            self.tp = OrcTpar(tau, x, y, scale, 1, *density, *sigt_range)

    def sigt_logd(self, s12, s13, sigt, p=None, grad=False):
        """log of the sigma_t density at each event (and its gradient in b0, b1, b2)."""
        p = self.p if p is None else _f64(p)
        s12, s13, sigt = (_f64(v) for v in (s12, s13, sigt))
        out = np.empty_like(s12)
        g = np.empty(3 * len(s12)) if grad else None
        _tddp_lib().orc_sigt_logd_many(C.byref(self.kin), C.byref(self.tp), _dp(p), len(s12),
                                        _dp(s12), _dp(s13), _dp(sigt), _dp(out),
                                        _dp(g) if grad else None)
        return (out, g.reshape(-1, 3)) if grad else out

    def _args(self, p):
        p = self.p if p is None else _f64(p)
        return (C.byref(self.kin), len(self.res), self._resarr(), C.byref(self.tp), _dp(p),
                len(p)), p

    def intensity_t(self, s12, s13, t, sigt, p=None):
        a, p = self._args(p)
        s12, s13, t, sigt = (_f64(v) for v in (s12, s13, t, sigt))
        out = np.empty_like(s12)
        _tddp_lib().orc_tddp_intensity(*a, len(s12), _dp(s12), _dp(s13), _dp(t), _dp(sigt),
                                       _dp(out))
        return out

    def norm_t(self, p=None, grad=False):
        a, p = self._args(p)
        dN = np.zeros(len(p)) if grad else None
        N = _tddp_lib().orc_tddp_norm(*a, self.nbx, self.nby, _dp(dN) if grad else None)
        return (N, dN) if grad else N

    def nll_t(self, s12, s13, t, sigt, p=None, grad=False):
        a, p = self._args(p)
        s12, s13, t, sigt = (_f64(v) for v in (s12, s13, t, sigt))
        out = np.zeros(1)
        g = np.zeros(len(p)) if grad else None
        _tddp_lib().orc_tddp_nll(*a, self.nbx, self.nby, len(s12), _dp(s12), _dp(s13), _dp(t),
                                 _dp(sigt), _dp(out), _dp(g) if grad else None)
        return (out[0], g) if grad else out[0]
