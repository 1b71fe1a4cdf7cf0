"""ctypes binding of ``libgoofit_gb.so`` (include/gf.h): argument marshalling only.

Every computation runs in the library's sm_103a kernels; this module converts numpy
arrays and Python lists to pointers and status codes to exceptions.  It never falls back
to a CPU path: if the library is missing or cannot load, the import of
``paper_1311_1753_gb300.gf`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

GF_OK, GF_EINVAL, GF_ENOMEM, GF_ECUDA, GF_ENONFINITE, GF_ENOCONV, GF_ETIMEOUT, GF_ESTATE = (
    0, -1, -2, -3, -4, -5, -6, -7)
GF_FP64, GF_MIXED = 0, 1
GF_METRIC_NLL, GF_METRIC_BINNED_NLL, GF_METRIC_CHISQ = 0, 1, 2

_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


class DalitzKin(C.Structure):
    _fields_ = [("M", C.c_double), ("m1", C.c_double), ("m2", C.c_double), ("m3", C.c_double),
                ("R", C.c_double)]


class Resonance(C.Structure):
    _fields_ = [("channel", C.c_int), ("spin", C.c_int), ("mass", C.c_int), ("width", C.c_int),
                ("re", C.c_int), ("im", C.c_int)]


class FitOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_calls", C.c_int), ("use_grad", C.c_int),
                ("up", C.c_double), ("hesse", C.c_int), ("refine", C.c_int)]


class FitResult(C.Structure):
    _fields_ = [("nll", C.c_double), ("edm", C.c_double), ("n_calls", C.c_int),
                ("n_iter", C.c_int), ("status", C.c_int), ("theta", _D), ("err", _D),
                ("cov", _D), ("n_calls_fast", C.c_int)]


class ServerOpts(C.Structure):
    _fields_ = [("device", C.c_int), ("precision", C.c_int), ("mem_budget", C.c_size_t),
                ("max_slots", C.c_int), ("wait_timeout_s", C.c_double)]


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        path = _build.build()
    lib = C.CDLL(path)
    vp = C.c_void_p
    sig = {
        "gf_create": ([C.POINTER(vp), C.c_int, C.c_int], C.c_int),
        "gf_destroy": ([vp], C.c_int),
        "gf_set_stream": ([vp, vp], C.c_int),
        "gf_strerror": ([C.c_int], C.c_char_p),
        "gf_last_error": ([vp, C.c_char_p, C.c_size_t], C.c_int),
        "gf_observable": ([vp, C.c_char_p, C.c_double, C.c_double, _I], C.c_int),
        "gf_parameter": ([vp, C.c_char_p, C.c_double, C.c_double, C.c_double, C.c_double, _I],
                         C.c_int),
        "gf_set_fixed": ([vp, C.c_int, C.c_int], C.c_int),
        "gf_set_value": ([vp, C.c_int, C.c_double], C.c_int),
        "gf_get_value": ([vp, C.c_int, _D], C.c_int),
        "gf_free_params": ([vp, _I, _I], C.c_int),
        "gf_pdf_exp": ([vp, C.c_int, C.c_int, _I], C.c_int),
        "gf_pdf_gauss": ([vp, C.c_int, C.c_int, C.c_int, _I], C.c_int),
        "gf_pdf_voigt": ([vp, C.c_int, C.c_int, C.c_int, C.c_int, _I], C.c_int),
        "gf_pdf_threshold": ([vp, C.c_int, C.c_int, C.c_int, C.c_int, _I], C.c_int),
        "gf_pdf_poly": ([vp, C.c_int, C.c_int, _I, _I], C.c_int),
        "gf_pdf_add": ([vp, C.c_int, _I, _I, _I], C.c_int),
        "gf_pdf_relbw": ([vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                          C.c_int, _I], C.c_int),
        "gf_pdf_conv": ([vp, C.c_int, C.c_int, C.c_int, _I], C.c_int),
        "gf_pdf_mapped": ([vp, C.c_int, C.c_int, _I, _I, _I], C.c_int),
        "gf_pdf_composite": ([vp, C.c_int, C.c_int, C.c_int, _I], C.c_int),
        "gf_pdf_prod": ([vp, C.c_int, _I, _I], C.c_int),
        "gf_pdf_dalitz": ([vp, C.c_int, C.c_int, C.POINTER(DalitzKin), C.c_int,
                           C.POINTER(Resonance), _I], C.c_int),
        "gf_set_norm_grid": ([vp, C.c_int, C.c_int, C.c_int], C.c_int),
        "gf_pdf_tddp": ([vp, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(DalitzKin), C.c_int,
                         C.POINTER(Resonance), C.c_int, C.c_int, C.c_int, C.c_int, _I], C.c_int),
        "gf_dalitz_inside": ([vp, C.c_int, C.c_int64, _D, _D, C.POINTER(C.c_int8)], C.c_int),
        "gf_dataset_create": ([vp, C.c_int, _I, C.POINTER(vp)], C.c_int),
        "gf_dataset_add_events": ([vp, C.c_int64, C.POINTER(_D)], C.c_int),
        "gf_dataset_create_binned": ([vp, C.c_int, _I, _I, _D, _D, C.POINTER(vp)], C.c_int),
        "gf_set_metric": ([vp, C.c_int], C.c_int),
        "gf_dataset_size": ([vp], C.c_int64),
        "gf_dataset_destroy": ([vp], C.c_int),
        "gf_set_data": ([vp, C.c_int, vp], C.c_int),
        "gf_set_data_device": ([vp, C.c_int, C.c_int, _I, C.c_int64, C.POINTER(vp)], C.c_int),
        "gf_nll": ([vp, _D, _D], C.c_int),
        "gf_nll_grad": ([vp, _D, _D, _D], C.c_int),
        "gf_nll_grad_start": ([vp, _D], C.c_int),
        "gf_nll_grad_finish": ([vp, _D, _D], C.c_int),
        "gf_logpdf": ([vp, _D, _D], C.c_int),
        "gf_logpdf_device": ([vp, _D, vp], C.c_int),
        "gf_dalitz_gram": ([vp, _D, _D], C.c_int),
        "gf_fit": ([vp, C.POINTER(FitOpts), C.POINTER(FitResult)], C.c_int),
        "gf_server_create": ([C.POINTER(ServerOpts), C.POINTER(vp)], C.c_int),
        "gf_server_submit": ([vp, vp, vp, C.c_int, C.POINTER(FitOpts), C.POINTER(C.c_uint64)],
                             C.c_int),
        "gf_server_poll": ([vp, C.c_uint64, C.POINTER(FitResult), _D, _I], C.c_int),
        "gf_server_nfree": ([vp, C.c_uint64, _I], C.c_int),
        "gf_server_drain": ([vp], C.c_int),
        "gf_server_stats": ([vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), _I], C.c_int),
        "gf_server_destroy": ([vp], C.c_int),
        "gf_last_eval_stats": ([vp, _D, _I], C.c_int),
        "gf_last_eval_times": ([vp, _D, _D], C.c_int),
        "gf_last_eval_graph": ([vp, _I, C.c_char_p, C.c_size_t], C.c_int),
        "gf_set_graphs": ([vp, C.c_int], C.c_int),
        "gf_set_event_sort": ([vp, C.c_int], C.c_int),
        "gf_set_mixture_path": ([vp, C.c_int], C.c_int),
        "gf_update_data": ([vp, C.c_int64, C.POINTER(_D)], C.c_int),
        "gf_prefetch_data": ([vp, C.c_int64, C.POINTER(_D)], C.c_int),
        "gf_nll_noalloc": ([vp, C.c_int, C.c_int, _I, C.c_int64, C.POINTER(vp), _D, vp], C.c_int),
        "gf_tddp_sigt_density": ([vp, C.c_int, C.c_int, C.c_int, C.c_int], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


class GFError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{lib.gf_strerror(code).decode()} ({code}){': ' + msg if msg else ''}")
        self.code = code


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Context:
    """A gf_ctx: observables, parameters, PDF nodes, data and evaluation."""

    def __init__(self, device: int = 0, precision: int = GF_FP64):
        self.h = C.c_void_p()
        rc = lib.gf_create(C.byref(self.h), device, precision)
        if rc:
            raise GFError(rc, "gf_create")
        self.precision = precision
        self._keep = []

    def close(self):
        if self.h:
            lib.gf_destroy(self.h)
            self.h = C.c_void_p()

    def release(self):
        """Give up ownership (e.g. to the fit server); the handle stays valid there."""
        h = self.h
        self.h = C.c_void_p()
        return h

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc, what=""):
        if rc != GF_OK:
            buf = C.create_string_buffer(512)
            if self.h:
                lib.gf_last_error(self.h, buf, 512)
            raise GFError(rc, f"{what}: {buf.value.decode()}")

    def _id(self, fn, *args):
        out = C.c_int(-1)
        self._ck(fn(self.h, *args, C.byref(out)), fn.__name__)
        return out.value

    # variables ------------------------------------------------------------------------
    def observable(self, name, lo, hi):
        return self._id(lib.gf_observable, name.encode(), lo, hi)

    def parameter(self, name, init, step, lo=0.0, hi=0.0, fixed=False):
        p = self._id(lib.gf_parameter, name.encode(), init, step, lo, hi)
        if fixed:
            self._ck(lib.gf_set_fixed(self.h, p, 1), "gf_set_fixed")
        return p

    def set_fixed(self, par, fixed=True):
        self._ck(lib.gf_set_fixed(self.h, par, 1 if fixed else 0), "gf_set_fixed")

    def set_value(self, par, v):
        self._ck(lib.gf_set_value(self.h, par, float(v)), "gf_set_value")

    def value(self, par):
        v = C.c_double()
        self._ck(lib.gf_get_value(self.h, par, C.byref(v)), "gf_get_value")
        return v.value

    def free_params(self):
        n = C.c_int()
        self._ck(lib.gf_free_params(self.h, C.byref(n), None), "gf_free_params")
        ids = (C.c_int * max(1, n.value))()
        self._ck(lib.gf_free_params(self.h, C.byref(n), ids), "gf_free_params")
        return list(ids)[: n.value]

    # nodes -------------------------------------------------------------------------------
    def exp(self, obs, alpha):
        return self._id(lib.gf_pdf_exp, obs, alpha)

    def gauss(self, obs, mu, sigma):
        return self._id(lib.gf_pdf_gauss, obs, mu, sigma)

    def voigt(self, obs, mu, sigma, width):
        return self._id(lib.gf_pdf_voigt, obs, mu, sigma, width)

    def threshold(self, obs, x0, power, c):
        return self._id(lib.gf_pdf_threshold, obs, x0, power, c)

    def poly(self, obs, coefs):
        arr = (C.c_int * len(coefs))(*coefs)
        return self._id(lib.gf_pdf_poly, obs, len(coefs), arr)

    def relbw(self, obs, dm0, gamma0, shift, ma, mb, radius, spin=1):
        """Relativistic Breit-Wigner line shape in x = m - shift (parameter ids; shift,
        ma, mb and radius fixed)."""
        return self._id(lib.gf_pdf_relbw, obs, dm0, gamma0, shift, ma, mb, radius, int(spin))

    def conv(self, obs, model, resolution, lattice=None):
        """ConvolutionPdf: model (over obs) convolved with resolution (over its own
        residual observable) on a lattice of `lattice` bins (default 1000)."""
        node = self._id(lib.gf_pdf_conv, obs, model, resolution)
        if lattice is not None:
            self.set_norm_grid(node, int(lattice))
        return node

    def mapped(self, obs, nodes, bounds):
        """MappedPdf: nodes[k] on [b_{k-1}, b_k); bounds = n - 1 fixed parameter ids."""
        n = (C.c_int * len(nodes))(*nodes)
        b = (C.c_int * max(1, len(bounds)))(*bounds)
        return self._id(lib.gf_pdf_mapped, obs, len(nodes), n, b)

    def composite(self, obs, core, shell):
        """CompositePdf: shell(core(x)), unnormalised shapes, normalised on obs's range."""
        return self._id(lib.gf_pdf_composite, obs, core, shell)

    def add(self, nodes, fracs):
        a = (C.c_int * len(nodes))(*nodes)
        f = (C.c_int * max(1, len(fracs)))(*fracs)
        return self._id(lib.gf_pdf_add, len(nodes), a, f)

    def prod(self, nodes):
        a = (C.c_int * len(nodes))(*nodes)
        return self._id(lib.gf_pdf_prod, len(nodes), a)

    def dalitz(self, obs12, obs13, kin: dict, resonances: list):
        k = DalitzKin(kin["M"], kin["m1"], kin["m2"], kin["m3"], kin.get("R", 1.5))
        rs = (Resonance * max(1, len(resonances)))(
            *[Resonance(r["channel"], r["spin"], r["mass"], r["width"], r["re"], r["im"])
              for r in resonances])
        return self._id(lib.gf_pdf_dalitz, obs12, obs13, C.byref(k), len(resonances), rs)

    def tddp(self, obs12, obs13, obs_t, obs_sigt, kin: dict, resonances: list, tau, x, y,
             scale):
        """Time-dependent Dalitz model (fixed resonance shapes); data columns s12, s13, t,
        sigma_t."""
        k = DalitzKin(kin["M"], kin["m1"], kin["m2"], kin["m3"], kin.get("R", 1.5))
        rs = (Resonance * max(1, len(resonances)))(
            *[Resonance(r["channel"], r["spin"], r["mass"], r["width"], r["re"], r["im"])
              for r in resonances])
        return self._id(lib.gf_pdf_tddp, obs12, obs13, obs_t, obs_sigt, C.byref(k),
                        len(resonances), rs, tau, x, y, scale)

    def tddp_sigt_density(self, node, b0, b1, b2):
        """gf_tddp_sigt_density: the sigma_t density (truncated Gamma(2), rate
        exp(b0 + b1 (s12 - sc) + b2 (s13 - sc))) of a time-dependent Dalitz node."""
        self._ck(lib.gf_tddp_sigt_density(self.h, node, b0, b1, b2), "gf_tddp_sigt_density")

    def set_norm_grid(self, node, nbx, nby=0):
        self._ck(lib.gf_set_norm_grid(self.h, node, nbx, nby), "gf_set_norm_grid")

    def dalitz_inside(self, node, s12, s13):
        s12, s13 = _f64(s12), _f64(s13)
        out = np.empty(len(s12), dtype=np.int8)
        self._ck(lib.gf_dalitz_inside(self.h, node, len(s12), _dp(s12), _dp(s13),
                                      out.ctypes.data_as(C.POINTER(C.c_int8))), "gf_dalitz_inside")
        return out.astype(bool)

    # data ----------------------------------------------------------------------------------
    def set_data(self, root, obs, cols):
        """Copy host columns (one per observable in ``obs``) to the device."""
        ds = C.c_void_p()
        ids = (C.c_int * len(obs))(*obs)
        self._ck(lib.gf_dataset_create(self.h, len(obs), ids, C.byref(ds)), "gf_dataset_create")
        try:
            cols = [_f64(c) for c in cols]
            ptrs = (_D * len(cols))(*[_dp(c) for c in cols])
            self._ck(lib.gf_dataset_add_events(ds, len(cols[0]), ptrs), "gf_dataset_add_events")
            self._ck(lib.gf_set_data(self.h, root, ds), "gf_set_data")
        finally:
            lib.gf_dataset_destroy(ds)
        self.n = len(cols[0])

    def make_dataset(self, obs, cols):
        """A host gf_dataset handle (for the fit server, which takes ownership)."""
        ds = C.c_void_p()
        ids = (C.c_int * len(obs))(*obs)
        self._ck(lib.gf_dataset_create(self.h, len(obs), ids, C.byref(ds)), "gf_dataset_create")
        cols = [_f64(c) for c in cols]
        ptrs = (_D * len(cols))(*[_dp(c) for c in cols])
        rc = lib.gf_dataset_add_events(ds, len(cols[0]), ptrs)
        if rc:
            lib.gf_dataset_destroy(ds)
            self._ck(rc, "gf_dataset_add_events")
        return ds

    def make_binned_dataset(self, obs, nbins, counts, errors=None):
        """A host binned gf_dataset: equal bins over each observable's range, contents
        row-major (last observable fastest), optional per-bin errors."""
        ds = C.c_void_p()
        ids = (C.c_int * len(obs))(*obs)
        nb = (C.c_int * len(obs))(*[int(b) for b in nbins])
        cnt = _f64(np.ravel(counts))
        err = _f64(np.ravel(errors)) if errors is not None else None
        self._ck(lib.gf_dataset_create_binned(self.h, len(obs), ids, nb, _dp(cnt),
                                              _dp(err) if err is not None else None,
                                              C.byref(ds)), "gf_dataset_create_binned")
        return ds

    def set_binned_data(self, root, obs, nbins, counts, errors=None):
        """Load a binned data set (bin centres as events, contents as weights)."""
        ds = self.make_binned_dataset(obs, nbins, counts, errors)
        try:
            self._ck(lib.gf_set_data(self.h, root, ds), "gf_set_data")
        finally:
            lib.gf_dataset_destroy(ds)
        self.n = int(np.prod(nbins))

    def set_metric(self, metric):
        self._ck(lib.gf_set_metric(self.h, int(metric)), "gf_set_metric")

    def set_data_device(self, root, obs, n, dev_ptrs, keep=None):
        """Use device columns in place (e.g. torch tensors' data_ptr()); ``keep`` holds
        the owning objects alive for the lifetime of this context."""
        ids = (C.c_int * len(obs))(*obs)
        ptrs = (C.c_void_p * len(dev_ptrs))(*dev_ptrs)
        self._ck(lib.gf_set_data_device(self.h, root, len(obs), ids, n, ptrs),
                 "gf_set_data_device")
        if keep is not None:
            self._keep.append(keep)
        self.n = n

    # evaluation ------------------------------------------------------------------------------
    def nll(self, theta):
        th = _f64(theta)
        out = C.c_double()
        rc = lib.gf_nll(self.h, _dp(th), C.byref(out))
        if rc == GF_ENONFINITE:
            return float("inf")
        self._ck(rc, "gf_nll")
        return out.value

    def nll_grad(self, theta):
        th = _f64(theta)
        out = C.c_double()
        g = np.zeros(len(th))
        rc = lib.gf_nll_grad(self.h, _dp(th), C.byref(out), _dp(g))
        if rc == GF_ENONFINITE:
            return float("inf"), g
        self._ck(rc, "gf_nll_grad")
        return out.value, g

    def nll_grad_start(self, theta):
        """gf_nll_grad_start: queue NLL + gradient at theta and return at once."""
        th = _f64(theta)
        self._ck(lib.gf_nll_grad_start(self.h, _dp(th)), "gf_nll_grad_start")
        self._nf_started = len(th)

    def nll_grad_finish(self):
        """gf_nll_grad_finish: wait for the started evaluation; (nll, gradient)."""
        out = C.c_double()
        g = np.zeros(getattr(self, "_nf_started", 0))
        rc = lib.gf_nll_grad_finish(self.h, C.byref(out), _dp(g))
        if rc == GF_ENONFINITE:
            return float("inf"), g
        self._ck(rc, "gf_nll_grad_finish")
        return out.value, g

    def logpdf(self, theta):
        th = _f64(theta)
        out = np.empty(self.n)
        self._ck(lib.gf_logpdf(self.h, _dp(th), _dp(out)), "gf_logpdf")
        return out

    def logpdf_device(self, theta, dev_ptr):
        th = _f64(theta)
        self._ck(lib.gf_logpdf_device(self.h, _dp(th), C.c_void_p(dev_ptr)), "gf_logpdf_device")

    def dalitz_gram(self, theta, nres):
        th = _f64(theta)
        G = np.zeros(2 * (nres + 1) ** 2)
        self._ck(lib.gf_dalitz_gram(self.h, _dp(th), _dp(G)), "gf_dalitz_gram")
        return (G[0::2] + 1j * G[1::2]).reshape(nres + 1, nres + 1)

    def set_stream(self, stream_ptr):
        self._ck(lib.gf_set_stream(self.h, C.c_void_p(stream_ptr)), "gf_set_stream")

    def update_data(self, cols):
        """Replace the loaded events (same n) from host columns; pinned arrays copy
        asynchronously.  Pass arrays that stay alive until the next evaluation."""
        ptrs = (_D * len(cols))(*[c.ctypes.data_as(_D) for c in cols])
        self._ck(lib.gf_update_data(self.h, len(cols[0]), ptrs), "gf_update_data")

    def update_data_ptrs(self, n, host_ptrs):
        ptrs = (_D * len(host_ptrs))(*[C.cast(C.c_void_p(p), _D) for p in host_ptrs])
        self._ck(lib.gf_update_data(self.h, n, ptrs), "gf_update_data")

    def prefetch_data_ptrs(self, n, host_ptrs):
        """gf_prefetch_data with raw host pointers (pinned buffers the caller keeps alive
        and unchanged until the gf_update_data that loads them)."""
        ptrs = (_D * len(host_ptrs))(*[C.cast(C.c_void_p(p), _D) for p in host_ptrs])
        self._ck(lib.gf_prefetch_data(self.h, n, ptrs), "gf_prefetch_data")

    def nll_noalloc(self, root, obs, n, dev_ptrs, theta, out_dev_ptr):
        """gf_nll_noalloc: NLL over caller-owned device columns into a caller-owned device
        double, with no allocation (queued on the context's stream)."""
        ids = (C.c_int * len(obs))(*obs)
        ptrs = (C.c_void_p * len(dev_ptrs))(*dev_ptrs)
        th = _f64(theta)
        self._ck(lib.gf_nll_noalloc(self.h, root, len(obs), ids, n, ptrs, _dp(th),
                                    C.c_void_p(out_dev_ptr)), "gf_nll_noalloc")

    def last_eval_times(self):
        t, s = C.c_double(), C.c_double()
        lib.gf_last_eval_times(self.h, C.byref(t), C.byref(s))
        return t.value, s.value

    def set_mixture_path(self, enable):
        self._ck(lib.gf_set_mixture_path(self.h, 1 if enable else 0), "gf_set_mixture_path")

    def set_event_sort(self, enable):
        self._ck(lib.gf_set_event_sort(self.h, 1 if enable else 0), "gf_set_event_sort")

    def set_graphs(self, enable):
        self._ck(lib.gf_set_graphs(self.h, 1 if enable else 0), "gf_set_graphs")

    def last_eval_graph(self):
        """(replayed, why_not): whether the last evaluation replayed a CUDA graph, and why
        graphs are off for this context if a capture failed ("" otherwise)."""
        r = C.c_int()
        buf = C.create_string_buffer(512)
        lib.gf_last_eval_graph(self.h, C.byref(r), buf, 512)
        return bool(r.value), buf.value.decode()

    def last_eval_stats(self):
        ms = C.c_double()
        nl = C.c_int()
        lib.gf_last_eval_stats(self.h, C.byref(ms), C.byref(nl))
        return ms.value, nl.value

    def fit(self, tol=1e-6, max_calls=5000, use_grad=True, up=0.0, hesse=True, refine=True):
        """up <= 0: the library's default for the metric (1 for chi-squared, else 0.5)."""
        nf = len(self.free_params())
        th = np.zeros(max(1, nf))
        err = np.zeros(max(1, nf))
        cov = np.zeros(max(1, nf * nf))
        o = FitOpts(tol, max_calls, 1 if use_grad else 0, up, 1 if hesse else 0,
                    1 if refine else 0)
        r = FitResult(0.0, 0.0, 0, 0, 0, _dp(th), _dp(err), _dp(cov), 0)
        rc = lib.gf_fit(self.h, C.byref(o), C.byref(r))
        if rc not in (GF_OK, GF_ENOCONV):
            self._ck(rc, "gf_fit")
        return dict(theta=th[:nf].copy(), err=err[:nf].copy(), cov=cov[: nf * nf].reshape(nf, nf),
                    nll=r.nll, edm=r.edm, n_calls=r.n_calls, n_iter=r.n_iter, status=r.status,
                    n_calls_fast=r.n_calls_fast)


class Server:
    """gf_server: continuous batching of many fits."""

    def __init__(self, device=0, precision=GF_MIXED, mem_budget=150 << 30, max_slots=64,
                 wait_timeout_s=120.0):
        self.h = C.c_void_p()
        o = ServerOpts(device, precision, mem_budget, max_slots, wait_timeout_s)
        rc = lib.gf_server_create(C.byref(o), C.byref(self.h))
        if rc:
            raise GFError(rc, "gf_server_create")

    def submit(self, ctx: Context, ds, root, tol=1e-6, max_calls=5000, hesse=True, refine=True):
        t = C.c_uint64()
        o = FitOpts(tol, max_calls, 1, 0.0, 1 if hesse else 0, 1 if refine else 0)
        rc = lib.gf_server_submit(self.h, ctx.h, ds, root, C.byref(o), C.byref(t))
        if rc:
            raise GFError(rc, "gf_server_submit")
        ctx.release()
        return t.value

    def poll(self, ticket):
        n = C.c_int()
        rc = lib.gf_server_nfree(self.h, ticket, C.byref(n))
        if rc:
            raise GFError(rc, "gf_server_nfree")
        nf = max(1, n.value)
        th, err = np.zeros(nf), np.zeros(nf)
        r = FitResult(0.0, 0.0, 0, 0, 0, _dp(th), _dp(err), None, 0)
        lat = C.c_double()
        done = C.c_int()
        rc = lib.gf_server_poll(self.h, ticket, C.byref(r), C.byref(lat), C.byref(done))
        if rc:
            raise GFError(rc, "gf_server_poll")
        if not done.value:
            return None
        return dict(theta=th[: n.value].copy(), err=err[: n.value].copy(), nll=r.nll, edm=r.edm,
                    n_calls=r.n_calls, n_calls_fast=r.n_calls_fast, status=r.status,
                    latency=lat.value)

    def drain(self):
        rc = lib.gf_server_drain(self.h)
        if rc:
            raise GFError(rc, "gf_server_drain")

    def stats(self):
        t, l, p = C.c_int64(), C.c_int64(), C.c_int()
        lib.gf_server_stats(self.h, C.byref(t), C.byref(l), C.byref(p))
        return dict(ticks=t.value, launches=l.value, peak_slots=p.value)

    def close(self):
        if self.h:
            lib.gf_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
