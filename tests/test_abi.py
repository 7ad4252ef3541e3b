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


def _params(**kw):
    from paper_2605_17869_gb300 import _abi
    p = _abi.SiftParams()
    _abi.load().sift_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_host_octave_geometry_equals_the_oracle(lib):
    """The library's host-side geometry (magnification decision and octave
    sizes, which size every launch and buffer) equals the oracle's, exactly,
    over random and boundary sizes and parameters; no device is needed."""
    import numpy as np
    import paper_2605_17869_gb300 as pkg
    from oracle import sift_oracle as so
    rng = np.random.default_rng(3)
    sizes = [(16, 16), (15, 400), (16, 17), (31, 32), (32, 31), (2000, 2000), (2000, 2001),
             (1, 1), (4000, 1000), (1000, 4000)]
    sizes += [tuple(int(v) for v in rng.integers(1, 5000, 2)) for _ in range(200)]
    for up, lim, ms in ((0, 4_000_000, 16), (1, 4_000_000, 16), (1, 0, 16), (1, 150 * 200, 16),
                        (1, 4_000_000, 40), (0, 4_000_000, 33)):
        p = _params(upsample=up, upsample_max_px=lim, min_octave_side=ms)
        op = so.Params(upsample=bool(up), upsample_max_px=lim, min_octave_side=ms)
        for H, W in sizes + [(150, 200), (150, 201), (4_000_000 // 2000, 2000)]:
            no, mag, geo = pkg.sift_octave_geometry(p, H, W)
            want = so.octave_sizes(H, W, op)
            assert mag == so.magnify(H, W, op), (up, lim, ms, H, W)
            assert no == len(want) and geo == [tuple(s) for s in want], (up, lim, ms, H, W)


def test_host_octave_geometry_argument_errors(lib):
    from paper_2605_17869_gb300 import _abi
    L = _abi.load()
    p = _params()
    no, mag = ctypes.c_int(), ctypes.c_int()
    hs = (ctypes.c_int * 4)()
    ok = L.sift_octave_geometry(ctypes.byref(p), 64, 64, ctypes.byref(no), ctypes.byref(mag), hs, hs, 4)
    assert ok == 0 and no.value == 3 and mag.value == 0 and hs[2] == 16
    assert L.sift_octave_geometry(None, 64, 64, ctypes.byref(no), ctypes.byref(mag), hs, hs, 4) \
        == _abi.SIFT_E_INVALID
    assert L.sift_octave_geometry(ctypes.byref(p), 0, 64, ctypes.byref(no), ctypes.byref(mag), hs, hs, 4) \
        == _abi.SIFT_E_INVALID
    assert L.sift_octave_geometry(ctypes.byref(p), 64, 64, ctypes.byref(no), ctypes.byref(mag), None, None, 4) \
        == _abi.SIFT_E_INVALID
    assert L.sift_octave_geometry(ctypes.byref(p), 64, 64, ctypes.byref(no), ctypes.byref(mag), None, None, 0) == 0
    bad = _params(n_scales=0)
    assert L.sift_octave_geometry(ctypes.byref(bad), 64, 64, ctypes.byref(no), ctypes.byref(mag), hs, hs, 4) \
        == _abi.SIFT_E_INVALID


def test_parameter_ranges_are_enforced_as_documented(lib):
    """Each documented parameter bound, on both sides, through the host-only
    geometry call (which validates like sift_create, without a device)."""
    from paper_2605_17869_gb300 import _abi
    L = _abi.load()
    no, mag = ctypes.c_int(), ctypes.c_int()

    def status(**kw):
        p = _params(**kw)
        return L.sift_octave_geometry(ctypes.byref(p), 64, 64, ctypes.byref(no), ctypes.byref(mag),
                                      None, None, 0)

    assert status() == 0
    nan = float("nan")
    for field, bad, good in (("n_scales", (1, 7), (3, 6)), ("sigma0", (0.0, -1.0, nan, 4.0), (1.0, 1.9)),
                             ("init_blur", (-0.1, nan), (0.0,)), ("contrast_thr", (0.0, nan), (1e-6,)),
                             ("edge_ratio", (0.0,), (1.0,)), ("prefilter_ratio", (-1.0, nan), (0.0,)),
                             ("ori_peak_ratio", (0.0, 1.01, nan), (1.0, 0.5)), ("border", (0,), (1,)),
                             ("max_refine_iter", (0,), (1,)), ("max_kpts", (0, -5), (1,)),
                             ("dsp", (2, -1), (0, 1)), ("upsample_max_px", (-1,), (0, 1)),
                             ("fp16_pyramid", (2, -1), (0, 1)),
                             ("min_octave_side", (15, 0), (16, 64))):
        for v in bad:
            assert status(**{field: v}) == _abi.SIFT_E_INVALID, (field, v)
        for v in good:
            assert status(**{field: v}) == 0, (field, v)
    # S = 2 at sigma0 = 1.6: the last level blur, 1.6 sqrt(2^4 - 2^3) = 4.5, needs
    # radius 19 > 16; at sigma0 = 1 it needs 12.
    assert status(n_scales=2) == _abi.SIFT_E_INVALID
    assert status(n_scales=2, sigma0=1.0) == 0
    # sigma0 = 2: the last level blur 2 sqrt(2^(10/3) - 2^(8/3)) = 3.86 needs radius
    # 16, so the octave side must exceed 16.
    assert status(sigma0=2.0) == _abi.SIFT_E_INVALID
    assert status(sigma0=2.0, min_octave_side=17) == 0
    assert status(border=8) == _abi.SIFT_E_INVALID               # 16 <= 2 x border
    assert status(border=8, min_octave_side=17) == 0


def _prototypes():
    """name -> parameter count, from the declarations in include/*.h."""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"(sift_\w+)\s*\(([^;{]*?)\)\s*;", src, re.S):
            args = m.group(2).strip()
            out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_arity_matches_the_header():
    from paper_2605_17869_gb300 import _abi
    protos = _prototypes()
    assert set(protos) == set(_abi.SIGNATURES)
    for name, (_, argtypes) in _abi.SIGNATURES.items():
        assert len(argtypes) == protos[name], name


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof and every field offset of the ABI structs, as a C compiler lays
    them out from the header, equal the ctypes mirrors."""
    import shutil
    import subprocess
    from paper_2605_17869_gb300 import _abi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"sift_params": _abi.SiftParams, "sift_kpts_dev": _abi.SiftKptsDev,
               "sift_result": _abi.SiftResult}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sift_gb300.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_binding_argument_types_match_the_header():
    """Each parameter's kind: pointers as pointers, and int, size_t, float,
    double, uint64_t and structs passed by value as exactly those ctypes."""
    from ctypes import c_char_p, c_double, c_float, c_int, c_size_t, c_uint64, c_void_p
    from paper_2605_17869_gb300 import _abi
    scalar = {"int": c_int, "size_t": c_size_t, "float": c_float, "double": c_double,
              "uint64_t": c_uint64, "sift_kpts_dev": _abi.SiftKptsDev, "sift_status": c_int}

    def is_ptr(t):
        return t in (c_void_p, c_char_p) or isinstance(t, type) and issubclass(t, ctypes._Pointer)

    seen = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"([\w\s\*]+?)\b(sift_\w+)\s*\(([^;{]*?)\)\s*;", src, re.S):
            ret, name, args = m.group(1).strip(), m.group(2), m.group(3).strip()
            seen.add(name)
            restype, argtypes = _abi.SIGNATURES[name]
            ret_t = ret.split()[-1] if "*" not in ret else "*"
            assert (is_ptr(restype) if ret_t == "*" else restype is scalar[ret_t]), name
            if args in ("", "void"):
                continue
            for k, a in enumerate(args.split(",")):
                a = " ".join(a.split())
                want_ptr = "*" in a
                base = re.sub(r"\bconst\b", "", a.replace("*", " ")).split()[0]
                got = argtypes[k]
                if want_ptr:
                    assert is_ptr(got), (name, k, a)
                else:
                    assert got is scalar[base], (name, k, a, got)
    assert seen == set(_abi.SIGNATURES)


def test_status_codes_match_the_header():
    from paper_2605_17869_gb300 import _abi
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "sift_gb300.h")).read(), flags=re.S)
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(SIFT_[A-Z_]+)\s*=\s*(-?\d+)", src)}
    assert len(codes) == 9
    for name, v in codes.items():
        assert getattr(_abi, name) == v, name
        assert _abi.STATUS_NAMES[v] == name


def test_binding_marshalling_on_cpu():
    """The batch marshalling of the binding: prebuilt ctypes arrays pass
    through, lists are converted, and images that are not 2-D float32 CUDA
    tensors with contiguous rows are refused before any library call."""
    import ctypes

    import paper_2605_17869_gb300 as pkg
    torch = pytest.importorskip("torch")
    arr = (ctypes.c_int * 3)(1, 2, 3)
    assert pkg._carray(ctypes.c_int, 3, arr) is arr
    assert list(pkg._carray(ctypes.c_int, 3, [4, 5, 6])) == [4, 5, 6]
    with pytest.raises(pkg.SiftError):
        pkg.Extractor._batch_dims([torch.zeros(4, 4)])  # on the host, not the device
