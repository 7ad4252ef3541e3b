"""The C-ABI library builds, loads without a GPU, and exports every entry
point declared in include/*.h (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_]\w*\s*\*?\s*(sift_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2605_17869_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_boundary():
    names = _declared()
    for need in ("sift_create", "sift_extract", "sift_extract_batch", "sift_serve_submit",
                 "sift_serve_poll", "sift_destroy", "sift_params_default"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_covers_every_symbol():
    from paper_2605_17869_gb300 import _abi
    assert _declared() == set(_abi.SIGNATURES)


def test_host_only_calls(lib):
    from paper_2605_17869_gb300 import _abi
    L = _abi.load()
    p = _abi.SiftParams()
    assert L.sift_params_default(ctypes.byref(p)) == 0
    assert (p.n_scales, p.max_refine_iter, p.border) == (3, 5, 5)
    assert abs(p.contrast_thr - 0.04 / 3) < 1e-7 and abs(p.sigma0 - 1.6) < 1e-7
    assert (p.upsample, p.upsample_max_px) == (0, 4_000_000)
    assert L.sift_version().startswith(b"gb300-sift")
    assert L.sift_params_default(None) == _abi.SIFT_E_INVALID
    h = ctypes.c_void_p()
    bad = _abi.SiftParams()
    L.sift_params_default(ctypes.byref(bad))
    bad.n_scales = 0
    assert L.sift_create(ctypes.byref(bad), ctypes.byref(h)) == _abi.SIFT_E_INVALID
    bad.n_scales, bad.sigma0 = 3, 4.0   # blur radius above 16
    assert L.sift_create(ctypes.byref(bad), ctypes.byref(h)) == _abi.SIFT_E_INVALID
    bad.sigma0, bad.upsample_max_px = 1.6, -1
    assert L.sift_create(ctypes.byref(bad), ctypes.byref(h)) == _abi.SIFT_E_INVALID
    assert L.sift_destroy(None) == _abi.SIFT_E_INVALID
    assert L.sift_serve_poll(None, 1, None) == _abi.SIFT_E_INVALID
