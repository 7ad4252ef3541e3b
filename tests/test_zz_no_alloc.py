"""sift_extract_noalloc: the allocation-free entry point against sift_extract.

The allocation-free variant exists for callers that cannot call cudaMalloc
(plug-ins whose host framework owns all device memory, real-time loops that
forbid allocation after start-up). It runs the same kernels on a fixed
in-library scratch array, so its output must equal sift_extract's bit for bit
(the tolerance used for GPU-vs-GPU comparisons throughout these tests). Calls
in a row on different images also check that nothing left in the shared
scratch by one call leaks into the next: a small image, then a larger one whose
layout covers everything the first wrote, then the small image again, whose
layout leaves part of the larger call's contents in place.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import pytest

from workloads import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_17869_gb300 as pkg  # noqa: E402
from paper_2605_17869_gb300 import _abi  # noqa: E402

K = 4096


def _noalloc(img, params):
    lib = _abi.load()
    buf = pkg.OutputBuffers(params.max_kpts, img.device)
    count = torch.zeros(1, dtype=torch.int32, device=img.device)
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.sift_extract_noalloc(ctypes.byref(params), ctypes.c_void_p(img.data_ptr()),
                                  img.shape[0], img.shape[1], img.stride(0),
                                  ctypes.c_void_p(stream), buf.kpts(),
                                  ctypes.c_void_p(buf.desc.data_ptr()),
                                  ctypes.c_void_p(count.data_ptr()))
    assert st == pkg.SIFT_OK, pkg.STATUS_NAMES.get(st, st)
    return buf.view(int(count.item()))


def _assert_same(a, b):
    assert a.count == b.count and a.count > 0
    for name in ("x", "y", "sigma", "angle", "response", "octave", "layer", "desc"):
        assert torch.equal(getattr(a, name), getattr(b, name)), name


def test_noalloc_matches_extract_two_calls_in_a_row():
    params = pkg.params(max_kpts=K)
    ex = pkg.Extractor(max_kpts=K)
    imgs = [torch.from_numpy(synth.single_vga(5)).cuda(),
            torch.from_numpy(synth.make_image(synth.rng_for(60, 0), 700, 900)).cuda()]
    refs = [ex.extract(im) for im in imgs]
    first = _noalloc(imgs[0], params)
    second = _noalloc(imgs[1], params)
    _assert_same(first, refs[0])
    _assert_same(second, refs[1])
    third = _noalloc(imgs[0], params)   # after the larger image: stale scratch beyond its layout
    _assert_same(third, refs[0])
    ex.close()


def test_noalloc_upsampled_and_limits():
    params = pkg.params(max_kpts=K, upsample=1)
    ex = pkg.Extractor(max_kpts=K, upsample=1)
    img = torch.from_numpy(synth.make_image(synth.rng_for(60, 1), 300, 400)).cuda()
    _assert_same(_noalloc(img, params), ex.extract(img))
    lib = _abi.load()
    big = torch.zeros((2000, 2000), device="cuda")
    buf = pkg.OutputBuffers(K, big.device)
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = lib.sift_extract_noalloc(ctypes.byref(params), ctypes.c_void_p(big.data_ptr()), 2000,
                                  2000, 2000, None, buf.kpts(),
                                  ctypes.c_void_p(buf.desc.data_ptr()),
                                  ctypes.c_void_p(count.data_ptr()))
    assert st == pkg.SIFT_E_BUDGET
    st = lib.sift_extract_noalloc(ctypes.byref(params), ctypes.c_void_p(big.data_ptr()), 15,
                                  2000, 2000, None, buf.kpts(),
                                  ctypes.c_void_p(buf.desc.data_ptr()),
                                  ctypes.c_void_p(count.data_ptr()))
    assert st == pkg.SIFT_E_INVALID
    ex.close()
