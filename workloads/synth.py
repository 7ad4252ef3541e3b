"""Seeded synthetic grayscale images shaped like the paper's benchmark workloads.

The paper evaluates on HPatches, IMC Phototourism and MegaDepth (§4.1), none
of which can be used here. These generators stand in for them: FP32
grayscale images in [0, 1] built from Gaussian blobs, rectangles, sinusoidal
gratings, optional 1/f texture and Gaussian noise, plus homography-warped
copies for the sequence / pair workloads.

This module is input generation only. It contains no part of the SIFT
computation, and both the FP64 oracle and the CUDA extractor consume its
output unchanged. Every image is a pure function of its seed
(NumPy PCG64, seed = workload index * 1000 + image index).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "make_image", "fractal_texture", "random_homography", "warp_homography",
    "single_vga", "homography_sequence", "wide_baseline_pair",
    "mixed_batch_shapes", "mixed_batch", "serving_trace", "rng_for",
]


def rng_for(workload: int, index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(workload * 1000 + index))


def fractal_texture(rng: np.random.Generator, h: int, w: int, std: float = 0.05) -> np.ndarray:
    """Zero-mean noise with a 1/f amplitude spectrum, scaled to the given std."""
    white = rng.standard_normal((h, w))
    spec = np.fft.rfft2(white)
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.rfftfreq(w)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    f[0, 0] = 1.0
    spec = spec / np.maximum(f, 1.0 / max(h, w))
    spec[0, 0] = 0.0
    tex = np.fft.irfft2(spec, s=(h, w))
    sd = tex.std()
    return tex * (std / sd) if sd > 0 else tex


def make_image(seed_rng: np.random.Generator, h: int, w: int, n_blobs: int = 40,
               n_rects: int = 10, n_gratings: int = 2, noise_std: float = 0.01,
               fractal_std: float = 0.0) -> np.ndarray:
    """Background 0.5 + blobs + rectangles + gratings (+ 1/f texture) + noise, clipped."""
    rng = seed_rng
    img = np.full((h, w), 0.5, dtype=np.float64)
    yy = np.arange(h, dtype=np.float64)
    xx = np.arange(w, dtype=np.float64)
    # Gaussian blobs: centre uniform, sigma log-uniform in [2, 30] px, amplitude in +-0.3.
    for _ in range(n_blobs):
        cx = rng.uniform(0, w)
        cy = rng.uniform(0, h)
        s = math.exp(rng.uniform(math.log(2.0), math.log(30.0)))
        a = rng.uniform(-0.3, 0.3)
        r = int(math.ceil(5 * s))
        x0, x1 = max(0, int(cx) - r), min(w, int(cx) + r + 1)
        y0, y1 = max(0, int(cy) - r), min(h, int(cy) + r + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        gx = np.exp(-((xx[x0:x1] - cx) ** 2) / (2 * s * s))
        gy = np.exp(-((yy[y0:y1] - cy) ** 2) / (2 * s * s))
        img[y0:y1, x0:x1] += a * np.outer(gy, gx)
    # Axis-aligned rectangles with an intensity offset in +-0.2.
    for _ in range(n_rects):
        xa, xb = np.sort(rng.integers(0, w, size=2))
        ya, yb = np.sort(rng.integers(0, h, size=2))
        img[ya:yb + 1, xa:xb + 1] += rng.uniform(-0.2, 0.2)
    # Sinusoidal gratings (period 8-64 px, amplitude 0.1) on a random disc.
    for _ in range(n_gratings):
        period = rng.uniform(8, 64)
        ang = rng.uniform(0, math.pi)
        phase = rng.uniform(0, 2 * math.pi)
        rad = rng.uniform(40, 150)
        cx = rng.uniform(0, w)
        cy = rng.uniform(0, h)
        x0, x1 = max(0, int(cx - rad)), min(w, int(cx + rad) + 1)
        y0, y1 = max(0, int(cy - rad)), min(h, int(cy + rad) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        X, Y = np.meshgrid(xx[x0:x1], yy[y0:y1])
        disc = (X - cx) ** 2 + (Y - cy) ** 2 <= rad * rad
        g = 0.1 * np.sin(2 * math.pi * (X * math.cos(ang) + Y * math.sin(ang)) / period + phase)
        img[y0:y1, x0:x1] += np.where(disc, g, 0.0)
    if fractal_std > 0:
        img += fractal_texture(rng, h, w, fractal_std)
    img += rng.normal(0.0, noise_std, size=(h, w))
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def random_homography(rng: np.random.Generator, h: int, w: int, max_rot_deg: float = 30.0,
                      scale_range=(0.6, 1.4), max_persp: float = 1e-4) -> np.ndarray:
    """3x3 homography about the image centre: rotation, isotropic scale, perspective."""
    th = math.radians(rng.uniform(-max_rot_deg, max_rot_deg))
    s = rng.uniform(*scale_range)
    p0, p1 = rng.uniform(-max_persp, max_persp, size=2)
    cx, cy = (w - 1) / 2.0, (h - 1) / 2.0
    A = np.array([[s * math.cos(th), -s * math.sin(th), 0.0],
                  [s * math.sin(th), s * math.cos(th), 0.0],
                  [p0, p1, 1.0]])
    T = np.array([[1.0, 0.0, cx], [0.0, 1.0, cy], [0.0, 0.0, 1.0]])
    Ti = np.array([[1.0, 0.0, -cx], [0.0, 1.0, -cy], [0.0, 0.0, 1.0]])
    return T @ A @ Ti


def warp_homography(src: np.ndarray, Hm: np.ndarray, fill: float = 0.5) -> np.ndarray:
    """dst(p) = src(Hm^-1 p), bilinear, out-of-bounds samples = fill."""
    h, w = src.shape
    Hi = np.linalg.inv(Hm)
    X, Y = np.meshgrid(np.arange(w, dtype=np.float64), np.arange(h, dtype=np.float64))
    den = Hi[2, 0] * X + Hi[2, 1] * Y + Hi[2, 2]
    sx = (Hi[0, 0] * X + Hi[0, 1] * Y + Hi[0, 2]) / den
    sy = (Hi[1, 0] * X + Hi[1, 1] * Y + Hi[1, 2]) / den
    x0 = np.floor(sx).astype(np.int64)
    y0 = np.floor(sy).astype(np.int64)
    fx = sx - x0
    fy = sy - y0
    s64 = src.astype(np.float64)

    def tap(yi, xi):
        ok = (xi >= 0) & (xi < w) & (yi >= 0) & (yi < h)
        v = s64[np.clip(yi, 0, h - 1), np.clip(xi, 0, w - 1)]
        return np.where(ok, v, fill)

    out = ((1 - fy) * ((1 - fx) * tap(y0, x0) + fx * tap(y0, x0 + 1))
           + fy * ((1 - fx) * tap(y0 + 1, x0) + fx * tap(y0 + 1, x0 + 1)))
    return out


# ---------------------------------------------------------------- workloads

def single_vga(index: int = 0) -> np.ndarray:
    """One 640x480 image (40 blobs, 10 rectangles, 2 gratings, N(0, 0.01) noise)."""
    return make_image(rng_for(0, index), 480, 640)


@dataclass
class Sequence:
    images: list
    homographies: list  # maps base-image pixel coords to image k coords (k >= 1)


def homography_sequence(index: int = 0, h: int = 750, w: int = 1000, n_warped: int = 5) -> Sequence:
    """A base image plus homography-warped, gain-scaled copies (HPatches-sequence shape)."""
    base = make_image(rng_for(1, index), h, w)
    rng = rng_for(1, 500 + index)
    imgs = [base]
    hs = [np.eye(3)]
    for _ in range(n_warped):
        Hm = random_homography(rng, h, w)
        gain = rng.uniform(0.7, 1.3)
        warped = np.clip(warp_homography(base, Hm) * gain, 0.0, 1.0).astype(np.float32)
        imgs.append(warped)
        hs.append(Hm)
    return Sequence(imgs, hs)


def wide_baseline_pair(index: int = 0, h: int = 1200, w: int = 1600) -> Sequence:
    """Two 1600x1200 images: textured base, and a warp of it with N(0, 0.02) noise."""
    base = make_image(rng_for(2, index), h, w, n_blobs=200, fractal_std=0.05)
    rng = rng_for(2, 500 + index)
    Hm = random_homography(rng, h, w)
    warped = warp_homography(base, Hm) + rng.normal(0.0, 0.02, size=(h, w))
    return Sequence([base, np.clip(warped, 0, 1).astype(np.float32)], [np.eye(3), Hm])


_ASPECTS = ((4, 3), (3, 4), (16, 9))


def mixed_batch_shapes(n: int = 64, index: int = 0):
    """(H, W) pairs: long side uniform in [480, 1600], aspect from {4:3, 3:4, 16:9}."""
    rng = rng_for(3, 900 + index)
    shapes = []
    for _ in range(n):
        long_side = int(rng.integers(480, 1601))
        a, b = _ASPECTS[int(rng.integers(0, 3))]
        if a >= b:  # landscape: width is the long side
            w, h = long_side, int(round(long_side * b / a))
        else:
            h, w = long_side, int(round(long_side * a / b))
        shapes.append((h, w))
    return shapes


def mixed_batch(n: int = 64, index: int = 0):
    """Mixed-resolution batch with 1/f texture (batching workload)."""
    return [make_image(rng_for(3, i), h, w, fractal_std=0.05)
            for i, (h, w) in enumerate(mixed_batch_shapes(n, index))]


_SERVE_RES = ((480, 640, 0.50), (1080, 1920, 0.35), (2160, 3840, 0.15))


def serving_trace(rate: float, n_requests: int, index: int = 0):
    """Poisson arrivals: list of (arrival time in s, H, W, image seed index)."""
    rng = rng_for(4, index)
    t = 0.0
    out = []
    probs = np.array([p for _, _, p in _SERVE_RES])
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        k = int(rng.choice(len(_SERVE_RES), p=probs))
        h, w, _ = _SERVE_RES[k]
        out.append((t, h, w, i))
    return out


def serving_image(h: int, w: int, seed_index: int) -> np.ndarray:
    return make_image(rng_for(4, 1000 + seed_index), h, w)
