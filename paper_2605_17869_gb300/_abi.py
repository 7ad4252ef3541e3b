"""ctypes declarations of the C ABI in include/sift_gb300.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_size_t, c_uint64, c_void_p

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsift_gb300.so")

SIFT_OK = 0
SIFT_W_TRUNCATED = 1
SIFT_PENDING = 2
SIFT_E_INVALID = -1
SIFT_E_OOM = -2
SIFT_E_CUDA = -3
SIFT_E_BUDGET = -4
SIFT_E_TIMEOUT = -5
SIFT_E_NOTFOUND = -6

STATUS_NAMES = {0: "SIFT_OK", 1: "SIFT_W_TRUNCATED", 2: "SIFT_PENDING", -1: "SIFT_E_INVALID",
                -2: "SIFT_E_OOM", -3: "SIFT_E_CUDA", -4: "SIFT_E_BUDGET", -5: "SIFT_E_TIMEOUT",
                -6: "SIFT_E_NOTFOUND"}


class SiftParams(ctypes.Structure):
    _fields_ = [("n_scales", c_int), ("sigma0", c_float), ("init_blur", c_float),
                ("upsample", c_int), ("min_octave_side", c_int), ("contrast_thr", c_float),
                ("edge_ratio", c_float), ("border", c_int), ("max_refine_iter", c_int),
                ("prefilter_ratio", c_float), ("ori_peak_ratio", c_float), ("max_kpts", c_int),
                ("upright", c_int), ("dsp", c_int), ("rootsift", c_int),
                ("upsample_max_px", c_int), ("fp16_pyramid", c_int)]


class SiftKptsDev(ctypes.Structure):
    _fields_ = [("x", c_void_p), ("y", c_void_p), ("sigma", c_void_p), ("angle", c_void_p),
                ("response", c_void_p), ("octave", c_void_p), ("layer", c_void_p)]


class SiftResult(ctypes.Structure):
    _fields_ = [("status", c_int), ("count", c_int), ("kpts", SiftKptsDev), ("desc", c_void_p),
                ("submit_to_done_ms", c_double)]


# name -> (restype, argtypes); every symbol declared in include/sift_gb300.h
SIGNATURES = {
    "sift_params_default": (c_int, [POINTER(SiftParams)]),
    "sift_create": (c_int, [POINTER(SiftParams), POINTER(c_void_p)]),
    "sift_destroy": (c_int, [c_void_p]),
    "sift_extract": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, SiftKptsDev,
                             c_void_p, c_void_p]),
    "sift_extract_batch": (c_int, [c_void_p, c_int, POINTER(c_void_p), POINTER(c_int),
                                   POINTER(c_int), POINTER(c_int), c_void_p,
                                   POINTER(SiftKptsDev), POINTER(c_void_p), c_void_p]),
    "sift_extract_noalloc": (c_int, [POINTER(SiftParams), c_void_p, c_int, c_int, c_int, c_void_p,
                                     SiftKptsDev, c_void_p, c_void_p]),
    "sift_match": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int, c_float, c_void_p,
                           c_void_p]),
    "sift_pack_outputs": (c_int, [c_void_p, c_void_p, c_void_p, c_size_t]),
    "sift_magsac": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_int, c_float, c_void_p,
                            c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sift_last_stats": (c_int, [c_void_p, POINTER(c_int), c_int]),
    "sift_pyramid_size": (c_int, [c_void_p, c_int, c_int, POINTER(c_int), POINTER(c_size_t)]),
    "sift_octave_geometry": (c_int, [POINTER(SiftParams), c_int, c_int, POINTER(c_int), POINTER(c_int),
                                     POINTER(c_int), POINTER(c_int), c_int]),
    "sift_build_pyramid": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p,
                                   c_size_t]),
    "sift_set_profiling": (c_int, [c_void_p, c_int]),
    "sift_kernel_times": (c_int, [c_void_p, POINTER(c_double), POINTER(c_int), c_int]),
    "sift_last_launch_count": (c_int, [c_void_p, POINTER(c_int)]),
    "sift_autotune": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "sift_get_tuning": (c_int, [c_void_p, c_char_p, c_size_t]),
    "sift_set_tuning": (c_int, [c_void_p, c_char_p]),
    "sift_autotune_batch": (c_int, [c_void_p, c_int, POINTER(c_void_p), POINTER(c_int),
                                    POINTER(c_int), POINTER(c_int), c_void_p,
                                    POINTER(SiftKptsDev), POINTER(c_void_p), c_void_p,
                                    POINTER(c_int)]),
    "sift_set_tuning_cache": (c_int, [c_void_p, c_char_p]),
    "sift_batch_signature": (c_int, [POINTER(SiftParams), c_int, POINTER(c_int), POINTER(c_int),
                                     c_char_p, c_size_t]),
    "sift_tuning_cache_get": (c_int, [c_char_p, c_char_p, c_char_p, c_size_t]),
    "sift_tuning_cache_put": (c_int, [c_char_p, c_char_p, c_char_p]),
    "sift_serve_create": (c_int, [c_void_p, c_size_t, c_int, POINTER(c_void_p)]),
    "sift_serve_submit": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, POINTER(c_uint64)]),
    "sift_serve_poll": (c_int, [c_void_p, c_uint64, POINTER(SiftResult)]),
    "sift_serve_wait": (c_int, [c_void_p, c_uint64, c_int, POINTER(SiftResult)]),
    "sift_serve_release": (c_int, [c_void_p, c_uint64]),
    "sift_serve_steps": (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_int), POINTER(c_double),
                                 POINTER(c_double), POINTER(c_int)]),
    "sift_serve_destroy": (c_int, [c_void_p]),
    "sift_last_error": (c_char_p, [c_void_p]),
    "sift_version": (c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build the CUDA extension first "
            "(python -m paper_2605_17869_gb300.build)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
