"""GPU-resident, bitwise-deterministic SIFT for NVIDIA GB300 (PySIFT, arXiv 2605.17869).

Python binding of the C ABI in include/sift_gb300.h. Every function named
`sift_*` here marshals its arguments into the library call of the same name;
every step of the extraction runs in the library's CUDA kernels. PyTorch is
used only to allocate device memory, name streams and hand results over by
DLPack (§3.3). There is no CPU fallback: if the compiled library is missing,
using this package raises.
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_double, c_float, c_int, c_size_t, c_uint64, c_void_p
from dataclasses import dataclass

from . import _abi
from ._abi import (SIFT_E_BUDGET, SIFT_E_CUDA, SIFT_E_INVALID, SIFT_E_NOTFOUND, SIFT_E_OOM,
                   SIFT_E_TIMEOUT, SIFT_OK, SIFT_PENDING, SIFT_W_TRUNCATED, STATUS_NAMES,
                   SiftKptsDev, SiftParams, SiftResult)

__all__ = [
    "SiftError", "SiftParams", "SiftKptsDev", "SiftResult", "Features", "Extractor", "Server",
    "sift_params_default", "sift_create", "sift_destroy", "sift_extract", "sift_extract_batch",
    "sift_extract_noalloc",
    "sift_last_stats", "sift_pyramid_size", "sift_octave_geometry", "sift_build_pyramid", "sift_set_profiling",
    "sift_kernel_times", "sift_last_launch_count", "sift_autotune", "sift_get_tuning", "sift_set_tuning",
    "sift_autotune_batch", "sift_set_tuning_cache", "sift_batch_signature", "sift_tuning_cache_get",
    "sift_tuning_cache_put",
    "sift_serve_create", "sift_serve_submit", "sift_serve_poll", "sift_serve_wait",
    "sift_serve_release", "sift_serve_steps", "sift_serve_destroy", "sift_last_error", "sift_version",
    "SIFT_OK", "SIFT_W_TRUNCATED", "SIFT_PENDING", "SIFT_E_INVALID", "SIFT_E_OOM",
    "SIFT_E_CUDA", "SIFT_E_BUDGET", "SIFT_E_TIMEOUT", "SIFT_E_NOTFOUND", "KERNEL_CLASSES",
]

KERNEL_CLASSES = ("blur", "base", "extrema", "decimate", "keypoint", "descriptor", "refine",
                  "orientation")


class SiftError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")


def _lib():
    return _abi.load()


def _check(st: int, handle=None, what: str = "") -> int:
    if st < 0:
        msg = what
        if handle is not None:
            msg = f"{what}: {_lib().sift_last_error(handle).decode()}"
        raise SiftError(st, msg)
    return st


# ------------------------------------------------------------ raw C ABI calls

def sift_version() -> str:
    return _lib().sift_version().decode()


def sift_params_default() -> SiftParams:
    p = SiftParams()
    _check(_lib().sift_params_default(byref(p)))
    return p


def sift_create(params: SiftParams) -> c_void_p:
    h = c_void_p()
    _check(_lib().sift_create(byref(params), byref(h)), what="sift_create")
    return h


def sift_destroy(handle) -> None:
    _check(_lib().sift_destroy(handle))


def sift_last_error(handle) -> str:
    return _lib().sift_last_error(handle).decode()


def sift_extract(handle, img_ptr: int, H: int, W: int, pitch: int, stream: int,
                 kpts: SiftKptsDev, desc_ptr: int, count_ptr: int) -> int:
    return _check(_lib().sift_extract(handle, c_void_p(img_ptr), H, W, pitch, c_void_p(stream),
                                      kpts, c_void_p(desc_ptr), c_void_p(count_ptr)),
                  handle, "sift_extract")


def _carray(ctype, n, xs):
    """xs as a ctypes array of n ctype; an array built beforehand passes through."""
    return xs if isinstance(xs, ctypes.Array) else (ctype * n)(*xs)


def sift_extract_batch(handle, img_ptrs, Hs, Ws, pitches, stream: int, kpts_list, desc_ptrs,
                       counts_ptr: int) -> int:
    n = len(img_ptrs)
    return _check(_lib().sift_extract_batch(
        handle, n, (c_void_p * n)(*img_ptrs), (c_int * n)(*Hs), (c_int * n)(*Ws),
        (c_int * n)(*pitches), c_void_p(stream), _carray(SiftKptsDev, n, kpts_list),
        _carray(c_void_p, n, desc_ptrs), c_void_p(counts_ptr)), handle, "sift_extract_batch")


def sift_extract_noalloc(params: SiftParams, img_ptr: int, H: int, W: int, pitch: int,
                         stream: int, kpts: SiftKptsDev, desc_ptr: int, count_ptr: int) -> int:
    """Allocation-free variant of sift_extract for callers that cannot call
    cudaMalloc (fixed 64 MiB in-library scratch; see the C header)."""
    return _check(_lib().sift_extract_noalloc(byref(params), c_void_p(img_ptr), H, W, pitch,
                                              c_void_p(stream), kpts, c_void_p(desc_ptr),
                                              c_void_p(count_ptr)), what="sift_extract_noalloc")


def sift_match(handle, a_ptr: int, n_a: int, b_ptr: int, n_b: int, ratio: float, stream: int,
               out_ptr: int) -> int:
    """Symmetric ratio-test matcher on fp16 tensor cores (see the C header)."""
    return _check(_lib().sift_match(handle, c_void_p(a_ptr), n_a, c_void_p(b_ptr), n_b,
                                    c_float(ratio), c_void_p(stream), c_void_p(out_ptr)),
                  handle, "sift_match")


def sift_magsac(handle, xa_ptr: int, xb_ptr: int, n: int, samples_ptr: int, n_hyp: int,
                sigma_max: float, stream: int, H_ptr: int, best_ptr: int, score_ptr: int,
                inliers_ptr: int, scores_ptr: int = 0) -> int:
    """GPU MAGSAC++ homography verification (see the C header)."""
    return _check(_lib().sift_magsac(handle, c_void_p(xa_ptr), c_void_p(xb_ptr), n,
                                     c_void_p(samples_ptr), n_hyp, c_float(sigma_max),
                                     c_void_p(stream), c_void_p(H_ptr), c_void_p(best_ptr),
                                     c_void_p(score_ptr), c_void_p(inliers_ptr),
                                     c_void_p(scores_ptr or None)),
                  handle, "sift_magsac")


def draw_samples(n: int, n_hyp: int = 1500, seed: int = 0):
    """Minimal samples for sift_magsac: an n_hyp x 4 int32 NumPy array of
    distinct indices in [0, n), each row uniform over the 4-subsets in draw
    order. Draw k picks uniformly among the n - k indices not yet taken (a
    value v is stepped past the taken indices in ascending order)."""
    import numpy as np
    if n < 4:
        raise SiftError(SIFT_E_INVALID, "MAGSAC++ needs at least 4 correspondences")
    rng = np.random.default_rng(seed)
    out = np.empty((n_hyp, 4), dtype=np.int64)
    for k in range(4):
        v = rng.integers(0, n - k, size=n_hyp)
        taken = np.sort(out[:, :k], axis=1)
        for j in range(k):
            v = v + (v >= taken[:, j])
        out[:, k] = v
    return out.astype(np.int32)


def sift_last_stats(handle, n_images: int):
    buf = (c_int * (4 * n_images))()
    st = _check(_lib().sift_last_stats(handle, buf, n_images), handle, "sift_last_stats")
    rows = [tuple(buf[4 * i:4 * i + 4]) for i in range(n_images)]
    return st, rows


def sift_pyramid_size(handle, H: int, W: int):
    no = c_int()
    tot = c_size_t()
    _check(_lib().sift_pyramid_size(handle, H, W, byref(no), byref(tot)), handle,
           "sift_pyramid_size")
    return no.value, tot.value


def sift_octave_geometry(params, H: int, W: int):
    """Host-only octave geometry: (n_octaves, magnified, [(H_o, W_o), ...])."""
    cap = 32
    no, mag = c_int(), c_int()
    hs, ws = (c_int * cap)(), (c_int * cap)()
    _check(_lib().sift_octave_geometry(byref(params), H, W, byref(no), byref(mag), hs, ws, cap),
           None, "sift_octave_geometry")
    n = min(no.value, cap)
    return no.value, bool(mag.value), [(hs[o], ws[o]) for o in range(n)]


def sift_build_pyramid(handle, img_ptr: int, H: int, W: int, pitch: int, stream: int,
                       out_ptr: int, out_elems: int) -> int:
    return _check(_lib().sift_build_pyramid(handle, c_void_p(img_ptr), H, W, pitch,
                                            c_void_p(stream), c_void_p(out_ptr), out_elems),
                  handle, "sift_build_pyramid")


def sift_set_profiling(handle, enable: bool) -> None:
    _check(_lib().sift_set_profiling(handle, int(bool(enable))), handle)


def sift_kernel_times(handle):
    n = len(KERNEL_CLASSES)
    ms = (c_double * n)()
    cnt = (c_int * n)()
    _check(_lib().sift_kernel_times(handle, ms, cnt, n), handle, "sift_kernel_times")
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_CLASSES)}


def sift_last_launch_count(handle) -> int:
    k = c_int()
    _check(_lib().sift_last_launch_count(handle, byref(k)), handle, "sift_last_launch_count")
    return k.value


def sift_autotune(handle, H: int, W: int, stream: int) -> None:
    _check(_lib().sift_autotune(handle, H, W, c_void_p(stream)), handle, "sift_autotune")


def sift_get_tuning(handle) -> str:
    buf = ctypes.create_string_buffer(4096)
    _check(_lib().sift_get_tuning(handle, buf, 4096), handle, "sift_get_tuning")
    return buf.value.decode()


def sift_set_tuning(handle, js: str) -> None:
    _check(_lib().sift_set_tuning(handle, js.encode()), handle, "sift_set_tuning")


def sift_autotune_batch(handle, img_ptrs, Hs, Ws, pitches, stream: int, kpts_list, desc_ptrs,
                        counts_ptr: int) -> bool:
    """Returns True when the tuning came from the handle's tuning cache."""
    n = len(img_ptrs)
    hit = c_int(0)
    _check(_lib().sift_autotune_batch(
        handle, n, (c_void_p * n)(*img_ptrs), (c_int * n)(*Hs), (c_int * n)(*Ws),
        (c_int * n)(*pitches), c_void_p(stream), _carray(SiftKptsDev, n, kpts_list),
        _carray(c_void_p, n, desc_ptrs), c_void_p(counts_ptr), byref(hit)), handle,
        "sift_autotune_batch")
    return bool(hit.value)


def sift_set_tuning_cache(handle, path) -> None:
    _check(_lib().sift_set_tuning_cache(handle, path.encode() if path else None), handle,
           "sift_set_tuning_cache")


def sift_batch_signature(params: SiftParams, Hs, Ws) -> str:
    n = len(Hs)
    buf = ctypes.create_string_buffer(1024)
    _check(_lib().sift_batch_signature(byref(params), n, (c_int * n)(*Hs), (c_int * n)(*Ws), buf,
                                       1024), None, "sift_batch_signature")
    return buf.value.decode()


def sift_tuning_cache_get(path: str, signature: str):
    """The stored tuning JSON, or None when the file or the entry is missing."""
    buf = ctypes.create_string_buffer(4096)
    st = _lib().sift_tuning_cache_get(path.encode(), signature.encode(), buf, 4096)
    if st == SIFT_E_NOTFOUND:
        return None
    _check(st, None, "sift_tuning_cache_get")
    return buf.value.decode()


def sift_tuning_cache_put(path: str, signature: str, js: str) -> None:
    _check(_lib().sift_tuning_cache_put(path.encode(), signature.encode(), js.encode()), None,
           "sift_tuning_cache_put")


def sift_serve_create(handle, budget_bytes: int, max_slots: int) -> c_void_p:
    s = c_void_p()
    _check(_lib().sift_serve_create(handle, budget_bytes, max_slots, byref(s)), handle,
           "sift_serve_create")
    return s


def sift_serve_submit(server, img_ptr: int, H: int, W: int, pitch: int) -> int:
    t = c_uint64()
    _check(_lib().sift_serve_submit(server, c_void_p(img_ptr), H, W, pitch, byref(t)),
           what="sift_serve_submit")
    return t.value


def sift_serve_poll(server, ticket: int):
    r = SiftResult()
    st = _lib().sift_serve_poll(server, ticket, byref(r))
    if st < 0:
        raise SiftError(st, "sift_serve_poll")
    return st, r


def sift_serve_wait(server, ticket: int, timeout_ms: int = 60000):
    r = SiftResult()
    st = _lib().sift_serve_wait(server, ticket, timeout_ms, byref(r))
    if st < 0:
        raise SiftError(st, "sift_serve_wait")
    return st, r


def sift_serve_release(server, ticket: int) -> None:
    _check(_lib().sift_serve_release(server, ticket), what="sift_serve_release")


def sift_serve_steps(server, max_steps: int = 65536):
    """Device-side intervals of the server's most recent finished steps, oldest
    first: a list of (lane, n_images, start_ms, end_ms)."""
    lane = (c_int * max_steps)()
    n_img = (c_int * max_steps)()
    t0 = (c_double * max_steps)()
    t1 = (c_double * max_steps)()
    n = c_int()
    _check(_lib().sift_serve_steps(server, max_steps, lane, n_img, t0, t1, byref(n)),
           what="sift_serve_steps")
    return [(lane[i], n_img[i], t0[i], t1[i]) for i in range(n.value)]


def sift_serve_destroy(server) -> None:
    _check(_lib().sift_serve_destroy(server), what="sift_serve_destroy")


# --------------------------------------------------------- torch-facing layer

def _torch():
    import torch  # noqa: PLC0415  (torch only provides memory, streams, DLPack)
    return torch


@dataclass
class Features:
    """Device-resident extraction result (torch CUDA tensors, length = count)."""
    x: object
    y: object
    sigma: object
    angle: object
    response: object
    octave: object
    layer: object
    desc: object
    count: int

    def as_numpy(self):
        return {k: getattr(self, k).cpu().numpy() for k in
                ("x", "y", "sigma", "angle", "response", "octave", "layer", "desc")}


class OutputBuffers:
    """Caller-owned output buffers for one image (capacity max_kpts)."""

    def __init__(self, max_kpts: int, device):
        torch = _torch()
        self.K = max_kpts
        f = dict(dtype=torch.float32, device=device)
        i = dict(dtype=torch.int32, device=device)
        self.x = torch.empty(max_kpts, **f)
        self.y = torch.empty(max_kpts, **f)
        self.sigma = torch.empty(max_kpts, **f)
        self.angle = torch.empty(max_kpts, **f)
        self.response = torch.empty(max_kpts, **f)
        self.octave = torch.empty(max_kpts, **i)
        self.layer = torch.empty(max_kpts, **i)
        self.desc = torch.empty((max_kpts, 128), **f)
        self._kpts = SiftKptsDev(self.x.data_ptr(), self.y.data_ptr(), self.sigma.data_ptr(),
                                 self.angle.data_ptr(), self.response.data_ptr(),
                                 self.octave.data_ptr(), self.layer.data_ptr())

    def kpts(self) -> SiftKptsDev:
        return self._kpts

    def view(self, n: int) -> Features:
        return Features(self.x[:n], self.y[:n], self.sigma[:n], self.angle[:n],
                        self.response[:n], self.octave[:n], self.layer[:n], self.desc[:n], n)


def params(**kw) -> SiftParams:
    p = sift_params_default()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown SIFT parameter {k!r}")
        setattr(p, k, v)
    return p


class Extractor:
    """One library handle plus reusable caller-owned output buffers.

    extract(img) and extract_batch(imgs) take float32 CUDA tensors (H x W,
    values in [0, 1]) and return device-resident Features. Work is queued on
    the current torch stream; `sync=True` waits for the counts.
    """

    def __init__(self, **kw):
        torch = _torch()
        if not torch.cuda.is_available():
            raise SiftError(SIFT_E_CUDA, "no CUDA device: the extractor runs only on the GPU")
        self.params = params(**kw)
        self.handle = sift_create(self.params)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._bufs = []
        self._out_arrays = {}  # n -> (SiftKptsDev[n], void*[n]) of the first n buffers
        self._counts = None
        self._last_batch = 0
        self._pack_dev = self._pack_host = self._counts_host = None

    def close(self):
        if getattr(self, "handle", None) is not None:
            _torch().cuda.synchronize()
            sift_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _buffers(self, n: int):
        torch = _torch()
        while len(self._bufs) < n:
            self._bufs.append(OutputBuffers(self.params.max_kpts, self.device))
        if self._counts is None or self._counts.numel() < n:
            self._counts = torch.zeros(max(n, 1), dtype=torch.int32, device=self.device)
        return self._bufs[:n]

    def _outputs(self, n: int):
        """The first n buffers and their pointer arrays, built once per n (the
        buffers live as long as the Extractor)."""
        bufs = self._buffers(n)
        arr = self._out_arrays.get(n)
        if arr is None:
            arr = ((SiftKptsDev * n)(*[b.kpts() for b in bufs]),
                   (c_void_p * n)(*[b.desc.data_ptr() for b in bufs]))
            self._out_arrays[n] = arr
        return bufs, arr

    @staticmethod
    def _check_img(img):
        torch = _torch()
        if not (img.is_cuda and img.dtype == torch.float32 and img.dim() == 2):
            raise SiftError(SIFT_E_INVALID, "image must be a 2-D float32 CUDA tensor")
        if img.stride(1) != 1:
            raise SiftError(SIFT_E_INVALID, "image rows must be contiguous")
        return img.shape[0], img.shape[1], img.stride(0)

    @staticmethod
    def _batch_dims(imgs):
        """(heights, widths, row pitches) of a batch, with _check_img's checks
        (one shape and one stride read per image: this runs on every call)."""
        f32 = _torch().float32
        Hs, Ws, Ps = [], [], []
        for img in imgs:
            sh, st = img.shape, img.stride()
            if not (img.is_cuda and img.dtype is f32 and len(sh) == 2):
                raise SiftError(SIFT_E_INVALID, "image must be a 2-D float32 CUDA tensor")
            if st[1] != 1:
                raise SiftError(SIFT_E_INVALID, "image rows must be contiguous")
            Hs.append(sh[0])
            Ws.append(sh[1])
            Ps.append(st[0])
        return Hs, Ws, Ps

    def extract_async(self, img, stream=None):
        """Queue one extraction; returns (buffers, counts tensor) without syncing."""
        torch = _torch()
        H, W, pitch = self._check_img(img)
        s = stream if stream is not None else torch.cuda.current_stream()
        buf = self._buffers(1)[0]
        sift_extract(self.handle, img.data_ptr(), H, W, pitch, s.cuda_stream, buf.kpts(),
                     buf.desc.data_ptr(), self._counts.data_ptr())
        self._last_batch = 1
        return buf, self._counts[:1]

    def extract(self, img, stream=None, copy: bool = True) -> Features:
        buf, cnt = self.extract_async(img, stream)
        n = int(cnt.item())
        f = buf.view(n)
        if copy:
            f = Features(*(t.clone() for t in (f.x, f.y, f.sigma, f.angle, f.response,
                                               f.octave, f.layer, f.desc)), n)
        return f

    def extract_batch_async(self, imgs, stream=None):
        torch = _torch()
        Hs, Ws, Ps = self._batch_dims(imgs)
        s = stream if stream is not None else torch.cuda.current_stream()
        bufs, (k_arr, d_arr) = self._outputs(len(imgs))
        sift_extract_batch(self.handle, [im.data_ptr() for im in imgs], Hs, Ws, Ps, s.cuda_stream,
                           k_arr, d_arr, self._counts.data_ptr())
        self._last_batch = len(imgs)
        return bufs, self._counts[:len(imgs)]

    def download(self, stream=None):
        """Bring the outputs of the last extract / extract_batch call to the host
        in one transfer. The library packs them on the device
        (sift_pack_outputs); the counts come back first, then exactly the packed
        bytes. Returns (counts, per-image list of dicts of NumPy arrays x, y,
        sigma, angle, response, octave, layer, desc); the arrays are views of a
        reused pinned buffer, valid until the next download. A batch of more than
        128 images runs as several launches and cannot be packed (SiftError);
        read its Features instead."""
        import numpy as np
        torch = _torch()
        n_img = self._last_batch
        if n_img < 1:
            raise SiftError(SIFT_E_INVALID, "no extraction to download")
        s = stream if stream is not None else torch.cuda.current_stream()
        rec = 128 * 4 + 7 * 4
        cap = n_img * self.params.max_kpts * rec
        if self._pack_dev is None or self._pack_dev.numel() < cap:
            self._pack_dev = torch.empty(cap, dtype=torch.uint8, device=self.device)
            self._pack_host = torch.empty(cap, dtype=torch.uint8).pin_memory()
        if self._counts_host is None or self._counts_host.numel() < n_img:
            self._counts_host = torch.empty(max(n_img, 128), dtype=torch.int32).pin_memory()
        _check(_lib().sift_pack_outputs(self.handle, c_void_p(s.cuda_stream),
                                        c_void_p(self._pack_dev.data_ptr()), c_size_t(cap)),
               self.handle, "sift_pack_outputs")
        with torch.cuda.stream(s):
            self._counts_host[:n_img].copy_(self._counts[:n_img], non_blocking=True)
            s.synchronize()
            counts = self._counts_host[:n_img].tolist()
            N = sum(counts)
            self._pack_host[:N * rec].copy_(self._pack_dev[:N * rec], non_blocking=True)
            s.synchronize()
        raw = self._pack_host.numpy()
        desc = raw[:N * 512].view(np.float32).reshape(N, 128)
        f = raw[N * 512:N * 532].view(np.float32).reshape(5, N)
        i = raw[N * 532:N * 540].view(np.int32).reshape(2, N)
        out, o = [], 0
        for n in counts:
            sl = slice(o, o + n)
            out.append({"x": f[0, sl], "y": f[1, sl], "sigma": f[2, sl], "angle": f[3, sl],
                        "response": f[4, sl], "octave": i[0, sl], "layer": i[1, sl],
                        "desc": desc[sl]})
            o += n
        return counts, out

    def extract_batch(self, imgs, stream=None, copy: bool = True):
        bufs, cnt = self.extract_batch_async(imgs, stream)
        counts = cnt.tolist()
        out = []
        for b, n in zip(bufs, counts):
            f = b.view(n)
            if copy:
                f = Features(*(t.clone() for t in (f.x, f.y, f.sigma, f.angle, f.response,
                                                   f.octave, f.layer, f.desc)), n)
            out.append(f)
        return out

    def match(self, desc_a, desc_b, ratio: float = 0.8, stream=None):
        """Mutual nearest neighbours of two descriptor sets (N x 128 float32 CUDA
        tensors) passing the ratio test both ways: an int32 tensor m with
        m[i] = j for each kept pair (i, j), else -1 (queued on the stream)."""
        torch = _torch()
        for t in (desc_a, desc_b):
            if not (t.is_cuda and t.dtype == torch.float32 and t.dim() == 2 and t.shape[1] == 128
                    and t.is_contiguous()):
                raise SiftError(SIFT_E_INVALID, "descriptors must be contiguous N x 128 float32 CUDA tensors")
        s = stream if stream is not None else torch.cuda.current_stream()
        out = torch.empty(desc_a.shape[0], dtype=torch.int32, device=desc_a.device)
        sift_match(self.handle, desc_a.data_ptr(), desc_a.shape[0], desc_b.data_ptr(),
                   desc_b.shape[0], ratio, s.cuda_stream, out.data_ptr())
        return out

    def magsac(self, xa, xb, samples=None, n_hyp: int = 1500, sigma_max: float = 1.0,
               seed: int = 0, stream=None):
        """GPU MAGSAC++ (§3.6): the best homography xa -> xb among n_hyp minimal
        samples (n x 2 float32 CUDA tensors of corresponding points). samples:
        an n_hyp x 4 int32 CUDA tensor, or None to draw them with draw_samples
        (seeded). Returns a dict of CUDA tensors, queued on the stream: H (3 x 3
        float64, H[2, 2] = 1), best (index, -1 if every sample is degenerate),
        score, inliers (n uint8), scores (n_hyp float32)."""
        torch = _torch()
        for t in (xa, xb):
            if not (t.is_cuda and t.dtype == torch.float32 and t.dim() == 2 and t.shape[1] == 2
                    and t.is_contiguous()):
                raise SiftError(SIFT_E_INVALID, "points must be contiguous N x 2 float32 CUDA tensors")
        n = xa.shape[0]
        if xb.shape[0] != n:
            raise SiftError(SIFT_E_INVALID, "xa and xb must have the same length")
        if samples is None:
            samples = torch.from_numpy(draw_samples(n, n_hyp, seed)).to(xa.device)
        if not (samples.is_cuda and samples.dtype == torch.int32 and samples.dim() == 2
                and samples.shape[1] == 4 and samples.is_contiguous()):
            raise SiftError(SIFT_E_INVALID, "samples must be a contiguous n_hyp x 4 int32 CUDA tensor")
        n_hyp = samples.shape[0]
        dev = xa.device
        out = {"H": torch.empty((3, 3), dtype=torch.float64, device=dev),
               "best": torch.empty(1, dtype=torch.int32, device=dev),
               "score": torch.empty(1, dtype=torch.float32, device=dev),
               "inliers": torch.empty(n, dtype=torch.uint8, device=dev),
               "scores": torch.empty(n_hyp, dtype=torch.float32, device=dev)}
        s = stream if stream is not None else torch.cuda.current_stream()
        sift_magsac(self.handle, xa.data_ptr(), xb.data_ptr(), n, samples.data_ptr(), n_hyp,
                    sigma_max, s.cuda_stream, out["H"].data_ptr(), out["best"].data_ptr(),
                    out["score"].data_ptr(), out["inliers"].data_ptr(), out["scores"].data_ptr())
        return out

    def stats(self, n_images: int = 1):
        return sift_last_stats(self.handle, n_images)

    def pyramid(self, img, stream=None):
        """Gaussian pyramid as a list (per octave) of (S+3, H_o, W_o) tensors."""
        torch = _torch()
        H, W, pitch = self._check_img(img)
        no, tot = sift_pyramid_size(self.handle, H, W)
        out = torch.empty(tot, dtype=torch.float32, device=self.device)
        s = stream if stream is not None else torch.cuda.current_stream()
        sift_build_pyramid(self.handle, img.data_ptr(), H, W, pitch, s.cuda_stream,
                           out.data_ptr(), tot)
        L = self.params.n_scales + 3
        lim = self.params.upsample_max_px
        up = bool(self.params.upsample) and (lim <= 0 or H * W <= lim)
        h = 2 * H if up else H
        w = 2 * W if up else W
        res, off = [], 0
        for _ in range(no):
            res.append(out[off:off + L * h * w].view(L, h, w))
            off += L * h * w
            h, w = h // 2, w // 2
        return res

    def set_profiling(self, on: bool):
        sift_set_profiling(self.handle, on)

    def kernel_times(self):
        return sift_kernel_times(self.handle)

    def launch_count(self) -> int:
        return sift_last_launch_count(self.handle)

    def autotune(self, H: int, W: int):
        sift_autotune(self.handle, H, W, _torch().cuda.current_stream().cuda_stream)
        return sift_get_tuning(self.handle)

    def autotune_batch(self, imgs, stream=None, cache=None):
        """Tune the launch shapes on this batch (sift_autotune_batch) and leave
        its results in the output buffers, like extract_batch_async. With
        cache (a file path), the tuning is looked up there first and stored
        there after a search. Returns (tuning JSON, whether it came from the
        cache)."""
        torch = _torch()
        Hs, Ws, Ps = self._batch_dims(imgs)
        s = stream if stream is not None else torch.cuda.current_stream()
        _, (k_arr, d_arr) = self._outputs(len(imgs))
        sift_set_tuning_cache(self.handle, cache)
        hit = sift_autotune_batch(self.handle, [im.data_ptr() for im in imgs], Hs, Ws, Ps,
                                  s.cuda_stream, k_arr, d_arr, self._counts.data_ptr())
        self._last_batch = len(imgs)
        return sift_get_tuning(self.handle), hit

    def get_tuning(self) -> str:
        return sift_get_tuning(self.handle)

    def set_tuning(self, js: str):
        sift_set_tuning(self.handle, js)


# ----------------------------------------------------------------- serving

class Server:
    """Continuous-batching server over an Extractor's parameters.

    submit() queues a device image and returns a ticket; result() waits and
    returns Features whose tensors are zero-copy DLPack views of the server's
    device buffers, valid until release(ticket).
    """

    def __init__(self, extractor: Extractor, budget_bytes: int = 8 << 30, max_slots: int = 64):
        self.ex = extractor
        self.K = extractor.params.max_kpts
        self.srv = sift_serve_create(extractor.handle, budget_bytes, max_slots)

    def submit(self, img) -> int:
        H, W, pitch = Extractor._check_img(img)
        return sift_serve_submit(self.srv, img.data_ptr(), H, W, pitch)

    def poll(self, ticket: int):
        st, r = sift_serve_poll(self.srv, ticket)
        return None if st == SIFT_PENDING else self._features(r)

    def result(self, ticket: int, timeout_ms: int = 60000):
        st, r = sift_serve_wait(self.srv, ticket, timeout_ms)
        return self._features(r), r.submit_to_done_ms, st

    def _features(self, r: SiftResult) -> Features:
        from ._dlpack import device_tensor
        n = r.count
        dev = self.ex.device.index
        k = r.kpts
        return Features(device_tensor(k.x, (n,), "f32", dev), device_tensor(k.y, (n,), "f32", dev),
                        device_tensor(k.sigma, (n,), "f32", dev),
                        device_tensor(k.angle, (n,), "f32", dev),
                        device_tensor(k.response, (n,), "f32", dev),
                        device_tensor(k.octave, (n,), "i32", dev),
                        device_tensor(k.layer, (n,), "i32", dev),
                        device_tensor(r.desc, (n, 128), "f32", dev), n)

    def release(self, ticket: int):
        sift_serve_release(self.srv, ticket)

    def steps(self, max_steps: int = 65536):
        """Device intervals of the most recent finished steps: (lane, n_images,
        start_ms, end_ms) each, oldest first (sift_serve_steps)."""
        return sift_serve_steps(self.srv, max_steps)

    def close(self):
        if getattr(self, "srv", None) is not None:
            sift_serve_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
