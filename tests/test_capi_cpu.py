"""C-ABI checks that need no GPU: the library builds and loads, every function that
include/gf.h declares is exported, status codes have text, and calls without a device
fail with a status instead of aborting."""
from __future__ import annotations

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("gf_create", "gf_destroy", "gf_observable", "gf_parameter", "gf_pdf_exp",
                 "gf_pdf_voigt", "gf_pdf_threshold", "gf_pdf_add", "gf_pdf_prod", "gf_pdf_dalitz",
                 "gf_dataset_create", "gf_dataset_add_events", "gf_set_data", "gf_nll",
                 "gf_nll_grad", "gf_fit", "gf_server_create", "gf_server_submit"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1311_1753_gb300 import _build
    lib = C.CDLL(_build.build())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_text_and_no_device_behaviour():
    from paper_1311_1753_gb300 import gf
    assert gf.lib.gf_strerror(gf.GF_ENONFINITE).decode().startswith("non-finite")
    assert gf.lib.gf_strerror(12345).decode() == "unknown status"
    h = C.c_void_p()
    rc = gf.lib.gf_create(C.byref(h), 0, 7)  # bad precision
    assert rc == gf.GF_EINVAL and not h.value
    rc = gf.lib.gf_create(C.byref(h), -1, gf.GF_FP64)
    assert rc in (gf.GF_ECUDA, gf.GF_EINVAL) and not h.value
    assert gf.lib.gf_destroy(None) == gf.GF_OK
    assert gf.lib.gf_nll(None, None, None) == gf.GF_EINVAL
    assert gf.lib.gf_nll_grad_start(None, None) == gf.GF_EINVAL
    assert gf.lib.gf_nll_grad_finish(None, None, None) == gf.GF_EINVAL
    assert gf.lib.gf_prefetch_data(None, 0, None) == gf.GF_EINVAL


def test_oracle_builds():
    import oracle
    assert os.path.exists(oracle.build())
