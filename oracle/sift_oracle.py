"""FP64 CPU oracle of the SIFT extraction path (test infrastructure only).

This module is the slow, plainly written reference that the CUDA extractor is
checked against. It is test infrastructure: only the test-suite, the smoke
check and the benchmark's CPU-baseline / reference arm may import it; the
product path never does, and it shares no code with the CUDA sources.

What it computes follows the paper's stage list (§3.2, "GPU Pipeline Stages"):
Gaussian scale space built by separable blurs with 4-sigma truncation, DoG
subtraction, 26-neighbour extrema with a contrast gate, sub-pixel refinement of
the 3-D Taylor expansion solved by Cramer's rule with up to five iterations and
Hessian edge rejection, 36-bin orientation histograms smoothed with
[1/4, 1/2, 1/4] and refined by a parabola, and 4x4x8 gradient descriptors with
the 0.2 clip and renormalisation: by default the plain single-scale form, and
optionally the DSP multi-scale pooling and RootSIFT normalisation of §3.2
("DSP Multi-Scale Descriptor Pooling", "RootSIFT Normalization"). Where the
paper is silent the textbook SIFT definition (Lowe, IJCV 2004, the method the
paper builds on, §1) is used; every such reading is marked READING below.

Arithmetic is float64 throughout. Each step is computed exactly as its
definition reads: no blocking, fusion or reordering beyond it.

Parity status per function:
  gaussian_taps, blur, upsample2x, decimate, store_level, build_pyramid, dog,
  find_candidates, refine_candidate, orientation_histogram,
  orientation_vote_margin, smooth_histogram, orientation_peaks,
  descriptor (plain, DSP and RootSIFT), normalise_descriptor,
  bilinear, cap_topk, magnify, for_image, octave_sizes : pinned by
  tests/test_oracle_pins.py (closed forms, brute force, invariants, rotation /
  transpose equivariance, hand-built DoG stacks and histograms), and the pins
  are themselves checked by planting mistakes (tests/test_oracle_mutations.py).
  extract (end-to-end composition): its level choice, decision margins, cap,
  upright mode, output scaling and blob scales are pinned; as an absolute
  result it is parity unpinned, since the paper prints no worked example.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np


# ------------------------------------------------------------------ parameters

@dataclass
class Params:
    n_scales: int = 3            # S, scales per octave (plain SIFT, 3)
    sigma0: float = 1.6          # base scale of each octave
    init_blur: float = 0.5       # blur assumed already present in the input
    upsample: bool = False       # first octave from a 2x magnified input (§5, double image)
    min_octave_side: int = 16    # keep octaves while min(H_o, W_o) >= this
    contrast_thr: float = 0.04 / 3
    edge_ratio: float = 10.0
    border: int = 5
    max_refine_iter: int = 5     # §3.2: five-iteration convergence
    prefilter_ratio: float = 0.5  # READING: pre-gate |D| > 0.5 * contrast_thr
    ori_bins: int = 36           # §3.2 table: 36-bin histogram
    ori_sigma_factor: float = 1.5
    ori_radius_factor: float = 3.0
    ori_peak_ratio: float = 0.8
    desc_width: int = 4          # 4x4 spatial cells
    desc_bins: int = 8           # 8 orientation bins -> 128-D
    desc_scale: float = 3.0      # spatial bin width = 3 sigma
    desc_clip: float = 0.2
    max_kpts: int = 0            # 0 = no cap
    upright: bool = False        # orientation fixed to 0 (no histogram)
    dsp: bool = False            # §3.2 DSP multi-scale descriptor pooling
    dsp_scales: tuple = (0.5, 2 ** -0.5, 1.0, 2 ** 0.5, 2.0)  # §3.2: 5 relative scales
    dsp_grid: int = 32           # §3.2: a 32 x 32 sample patch per DSP scale
    rootsift: bool = False       # §3.2 RootSIFT: L1 normalise, then element-wise sqrt
    upsample_max_px: int = 4_000_000  # §5: no magnification above 4 MP (0 = no limit)
    fp16_pyramid: bool = False   # §3.2: levels of octaves above 0 stored in fp16, octave 0 in full precision


# ------------------------------------------------------------------ A2/A3: blur

def gaussian_taps(sigma: float):
    """Sampled Gaussian with 4-sigma truncation (§3.2), normalised to sum 1.

    READING: radius r = ceil(4 sigma); taps w_k = exp(-k^2 / (2 sigma^2)) for
    k = -r..r, divided by their sum.
    """
    r = int(math.ceil(4.0 * sigma))
    k = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-(k * k) / (2.0 * sigma * sigma))
    return r, w / w.sum()


def _pad_reflect101(a: np.ndarray, r: int, axis: int) -> np.ndarray:
    """READING: border mode reflect-101 (index -k -> k, n-1+k -> n-1-k)."""
    pad = [(0, 0)] * a.ndim
    pad[axis] = (r, r)
    return np.pad(a, pad, mode="reflect")  # numpy 'reflect' excludes the edge sample


def blur(img: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian convolution (§3.2): a row pass, then a column pass."""
    r, w = gaussian_taps(sigma)
    h, wd = img.shape
    p = _pad_reflect101(img.astype(np.float64), r, axis=1)
    rows = np.zeros((h, wd))
    for j in range(2 * r + 1):
        rows += w[j] * p[:, j:j + wd]
    p = _pad_reflect101(rows, r, axis=0)
    out = np.zeros((h, wd))
    for j in range(2 * r + 1):
        out += w[j] * p[j:j + h, :]
    return out


# ------------------------------------------------------------ A1/A4: resampling

def upsample2x(img: np.ndarray) -> np.ndarray:
    """READING of the 2x magnified first octave (§5): u[2k] = I[k],
    u[2k+1] = (I[k] + I[k+1]) / 2 with the last sample clamped, in both axes."""
    def up1(a, axis):
        a = np.moveaxis(a, axis, 0)
        n = a.shape[0]
        out = np.empty((2 * n,) + a.shape[1:])
        nxt = np.concatenate([a[1:], a[-1:]], axis=0)
        out[0::2] = a
        out[1::2] = 0.5 * (a + nxt)
        return np.moveaxis(out, 0, axis)
    return up1(up1(img.astype(np.float64), 1), 0)


def decimate(img: np.ndarray) -> np.ndarray:
    """READING: next octave base = every second sample of level S, size floor(n/2)."""
    h, w = img.shape
    return img[0:2 * (h // 2):2, 0:2 * (w // 2):2].copy()


# ------------------------------------------------------------------ pyramid

def magnify(h: int, w: int, p: Params) -> bool:
    """Whether an h x w input gets the 2x magnified first octave. The paper's
    VRAM-adaptive execution (§1 contributions, §5 "Resolution Scaling")
    suppresses the double image above 4 MP. READING: the limit counts input
    pixels, an image of exactly upsample_max_px pixels is still magnified, and
    0 turns the limit off."""
    return bool(p.upsample) and (p.upsample_max_px <= 0 or h * w <= p.upsample_max_px)


def for_image(h: int, w: int, p: Params) -> Params:
    """The parameters one h x w image is processed with: upsample resolved by
    magnify(); every later step reads only this resolved flag."""
    up = magnify(h, w, p)
    return p if up == bool(p.upsample) else replace(p, upsample=up)


def octave_sizes(h: int, w: int, p: Params):
    """Octave geometry: (H_o, W_o) while min side >= min_octave_side."""
    if magnify(h, w, p):
        h, w = 2 * h, 2 * w
    sizes = []
    while min(h, w) >= p.min_octave_side:
        sizes.append((h, w))
        h, w = h // 2, w // 2
    return sizes


def level_sigmas(p: Params):
    """Nominal octave-relative scales sigma_i = sigma0 * 2^(i/S), i = 0..S+2."""
    return [p.sigma0 * 2.0 ** (i / p.n_scales) for i in range(p.n_scales + 3)]


def increment_sigmas(p: Params):
    """kappa_i = sqrt(sigma_i^2 - sigma_{i-1}^2): blur taking level i-1 to level i."""
    s = level_sigmas(p)
    return [math.sqrt(s[i] ** 2 - s[i - 1] ** 2) for i in range(1, len(s))]


def base_sigma(p: Params) -> float:
    """Blur that brings the (possibly magnified) input to sigma0."""
    eff = p.init_blur * (2.0 if p.upsample else 1.0)
    d = p.sigma0 ** 2 - eff ** 2
    return math.sqrt(d) if d > 0 else 0.0


def store_level(level: np.ndarray, o: int, p: Params) -> np.ndarray:
    """The value a pyramid level keeps once stored (§3.2, "fp16 storage with fp32
    compute (octave 0 in fp32)"). READING: with fp16_pyramid, every level of an
    octave above 0 is rounded to the nearest IEEE binary16 value (ties to even)
    as soon as it is formed, and the next level (and the next octave's
    decimated base) is computed from the rounded values; octave 0 and the
    default mode keep full precision."""
    if p.fp16_pyramid and o > 0:
        return level.astype(np.float16).astype(np.float64)
    return level


def build_pyramid(img: np.ndarray, p: Params):
    """Gaussian scale space (§3.2): per octave S+3 levels, each level blurred from
    the previous one (READING of the paper's in-place construction, §4.2).
    With fp16_pyramid every level of octaves above 0 is stored in fp16
    (store_level)."""
    img = np.asarray(img, dtype=np.float64)
    p = for_image(img.shape[0], img.shape[1], p)
    base = upsample2x(img) if p.upsample else img
    sb = base_sigma(p)
    kap = increment_sigmas(p)
    sizes = octave_sizes(img.shape[0], img.shape[1], p)
    octaves = []
    for o, (h, w) in enumerate(sizes):
        if o == 0:
            g0 = blur(base, sb) if sb > 0 else base.copy()
        else:
            g0 = decimate(octaves[o - 1][p.n_scales])
        assert g0.shape == (h, w)
        levels = [store_level(g0, o, p)]
        for k in kap:
            levels.append(store_level(blur(levels[-1], k), o, p))
        octaves.append(np.stack(levels))
    return octaves


def dog(octave: np.ndarray) -> np.ndarray:
    """Difference of Gaussians D_i = G_{i+1} - G_i (§3.2)."""
    return octave[1:] - octave[:-1]


# ------------------------------------------------------------------ A5: extrema

def find_candidates(D: np.ndarray, p: Params):
    """3x3x3 extrema with contrast gating (§3.2).

    READING: layers s = 1..S, border b <= x < W-b and b <= y < H-b, pre-gate
    |D| > prefilter_ratio * contrast_thr, and D strictly above all 26 neighbours
    or strictly below all of them. Returns (s, y, x) in (s, y, x) order plus the
    two relative decision margins (pre-gate, and smallest neighbour gap / |D|).
    """
    S = p.n_scales
    b = p.border
    _, h, w = D.shape
    out_s, out_y, out_x, m_gate, m_ext = [], [], [], [], []
    if h - 2 * b <= 0 or w - 2 * b <= 0:
        z = np.zeros(0, dtype=np.int64)
        return z, z, z, np.zeros(0), np.zeros(0)
    thr = p.prefilter_ratio * p.contrast_thr
    for s in range(1, S + 1):
        c = D[s, b:h - b, b:w - b]
        nmax = np.full(c.shape, -np.inf)
        nmin = np.full(c.shape, np.inf)
        for ds in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if ds == 0 and dy == 0 and dx == 0:
                        continue
                    n = D[s + ds, b + dy:h - b + dy, b + dx:w - b + dx]
                    nmax = np.maximum(nmax, n)
                    nmin = np.minimum(nmin, n)
        is_max = c > nmax
        is_min = c < nmin
        gate = np.abs(c) > thr
        ys, xs = np.nonzero(gate & (is_max | is_min))
        cv = c[ys, xs]
        gap = np.where(is_max[ys, xs], cv - nmax[ys, xs], nmin[ys, xs] - cv)
        out_s.append(np.full(len(ys), s))
        out_y.append(ys + b)
        out_x.append(xs + b)
        m_gate.append((np.abs(cv) - thr) / np.maximum(np.abs(cv), thr))
        m_ext.append(gap / np.abs(cv))
    return (np.concatenate(out_s), np.concatenate(out_y), np.concatenate(out_x),
            np.concatenate(m_gate), np.concatenate(m_ext))


# --------------------------------------------------------------- A6: refinement

def _round_half_away(v: float) -> int:
    return int(math.floor(abs(v) + 0.5)) * (1 if v >= 0 else -1)


def derivatives(D: np.ndarray, s: int, y: int, x: int):
    """Gradient and Hessian of D at (x, y, s) by central differences."""
    c = D[s, y, x]
    dx = 0.5 * (D[s, y, x + 1] - D[s, y, x - 1])
    dy = 0.5 * (D[s, y + 1, x] - D[s, y - 1, x])
    ds = 0.5 * (D[s + 1, y, x] - D[s - 1, y, x])
    dxx = D[s, y, x + 1] + D[s, y, x - 1] - 2.0 * c
    dyy = D[s, y + 1, x] + D[s, y - 1, x] - 2.0 * c
    dss = D[s + 1, y, x] + D[s - 1, y, x] - 2.0 * c
    dxy = 0.25 * (D[s, y + 1, x + 1] - D[s, y + 1, x - 1] - D[s, y - 1, x + 1] + D[s, y - 1, x - 1])
    dxs = 0.25 * (D[s + 1, y, x + 1] - D[s + 1, y, x - 1] - D[s - 1, y, x + 1] + D[s - 1, y, x - 1])
    dys = 0.25 * (D[s + 1, y + 1, x] - D[s + 1, y - 1, x] - D[s - 1, y + 1, x] + D[s - 1, y - 1, x])
    g = np.array([dx, dy, ds])
    H = np.array([[dxx, dxy, dxs], [dxy, dyy, dys], [dxs, dys, dss]])
    return g, H


def det3(M) -> float:
    return (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
            - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
            + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]))


def cramer_solve(H: np.ndarray, rhs: np.ndarray):
    """Solve H v = rhs by Cramer's rule (§3.2); None when det H == 0."""
    d = det3(H)
    if d == 0.0:
        return None
    v = np.empty(3)
    for k in range(3):
        M = H.copy()
        M[:, k] = rhs
        v[k] = det3(M) / d
    return v


# Rejection codes, shared meaning with the CUDA side's debug output.
KEEP, REJ_SINGULAR, REJ_NOCONV, REJ_BOUNDS, REJ_CONTRAST, REJ_EDGE = 0, 1, 2, 3, 4, 5


@dataclass
class Refined:
    code: int
    x: int = 0
    y: int = 0
    s: int = 0
    dx: float = 0.0
    dy: float = 0.0
    ds: float = 0.0
    response: float = 0.0
    margin: float = math.inf


def refine_candidate(D: np.ndarray, s: int, y: int, x: int, p: Params) -> Refined:
    """Sub-pixel refinement of one candidate (§3.2).

    READING (textbook SIFT): up to max_refine_iter steps; at each, solve
    H delta = -g by Cramer; converged when max|delta| < 0.5; otherwise move the
    integer position by delta rounded half away from zero, rejecting moves that
    leave the border band or the layer range 1..S. Then the interpolated
    contrast |D + g.delta/2| must be >= contrast_thr, and the spatial Hessian
    must pass tr^2 * r < (r+1)^2 * det with det > 0.
    The returned margin is the smallest relative distance of any of these
    decisions from its threshold, |a - t| / max(|a|, |t|).
    """
    S = p.n_scales
    b = p.border
    _, h, w = D.shape
    margin = math.inf
    delta = None
    for _ in range(p.max_refine_iter):
        g, H = derivatives(D, s, y, x)
        delta = cramer_solve(H, -g)
        if delta is None or not np.all(np.isfinite(delta)):
            return Refined(REJ_SINGULAR, margin=margin)
        m = float(np.max(np.abs(delta)))
        margin = min(margin, abs(0.5 - m) / 0.5)
        if m < 0.5:
            break
        for v in delta:
            a = abs(v)
            edge = math.floor(a) + 0.5
            margin = min(margin, abs(a - edge) / edge)
        if m > 1e7:  # far outside any image: same outcome as the bounds check
            return Refined(REJ_BOUNDS, margin=margin)
        x += _round_half_away(delta[0])
        y += _round_half_away(delta[1])
        s += _round_half_away(delta[2])
        if s < 1 or s > S or x < b or x >= w - b or y < b or y >= h - b:
            return Refined(REJ_BOUNDS, margin=margin)
    else:
        return Refined(REJ_NOCONV, margin=margin)
    g, H = derivatives(D, s, y, x)
    contrast = D[s, y, x] + 0.5 * float(g @ delta)
    margin = min(margin, abs(abs(contrast) - p.contrast_thr) / max(abs(contrast), p.contrast_thr))
    if abs(contrast) < p.contrast_thr:
        return Refined(REJ_CONTRAST, margin=margin)
    dxx, dyy, dxy = H[0, 0], H[1, 1], H[0, 1]
    tr = dxx + dyy
    det = dxx * dyy - dxy * dxy
    r = p.edge_ratio
    lhs, rhs = tr * tr * r, (r + 1) ** 2 * det
    denom = abs(lhs) + abs(rhs)
    if denom > 0:
        margin = min(margin, abs(rhs - lhs) / denom)
    if det <= 0 or lhs >= rhs:
        return Refined(REJ_EDGE, margin=margin)
    return Refined(KEEP, x, y, s, float(delta[0]), float(delta[1]), float(delta[2]),
                   abs(contrast), margin)


# --------------------------------------------------------------- A7: orientation

def _gradients(L: np.ndarray, ys: np.ndarray, xs: np.ndarray):
    """dx = L(x+1) - L(x-1), dy = L(y+1) - L(y-1) (y pointing down)."""
    dx = L[ys, xs + 1] - L[ys, xs - 1]
    dy = L[ys + 1, xs] - L[ys - 1, xs]
    return dx, dy


def _round_pos(v: float) -> int:
    return int(math.floor(v + 0.5))


def orientation_histogram(L: np.ndarray, xi: int, yi: int, sigma_oct: float, p: Params):
    """Raw 36-bin gradient-orientation histogram around an integer pixel (§3.2).

    READING: Gaussian window sigma_w = 1.5 sigma, square radius round(3 sigma_w),
    samples with 1 <= x <= W-2 and 1 <= y <= H-2, weight m * exp(-(i^2+j^2) /
    (2 sigma_w^2)) with (i, j) the integer offset, nearest-bin voting
    floor(n theta / 2 pi + 1/2). A gradient with |dx| = |dy| (theta an odd
    multiple of 45 degrees, the only bin boundaries a gradient can hit exactly)
    is decided exactly by that formula in integers: (n (2q + 1) + 4) // 8 for
    quadrant q, so a half-bin value goes up.
    """
    h, w = L.shape
    n = p.ori_bins
    sw = p.ori_sigma_factor * sigma_oct
    R = _round_pos(p.ori_radius_factor * sw)
    j, i = np.meshgrid(np.arange(-R, R + 1), np.arange(-R, R + 1), indexing="ij")
    ys, xs = yi + j, xi + i
    ok = (xs >= 1) & (xs <= w - 2) & (ys >= 1) & (ys <= h - 2)
    ys, xs, i, j = ys[ok], xs[ok], i[ok], j[ok]
    dx, dy = _gradients(L, ys, xs)
    mag = np.sqrt(dx * dx + dy * dy)
    th = np.arctan2(dy, dx)
    th = np.where(th < 0, th + 2 * math.pi, th)
    wt = np.exp(-(i * i + j * j) / (2.0 * sw * sw))
    bins = np.floor(n * th / (2 * math.pi) + 0.5).astype(np.int64) % n
    diag, q = _diagonal_quadrant(dx, dy)
    bins = np.where(diag, (n * (2 * q + 1) + 4) // 8 % n, bins)
    return np.bincount(bins, weights=wt * mag, minlength=n)


def _diagonal_quadrant(dx, dy):
    """Gradients with |dx| = |dy| != 0 and their quadrant q (theta = 45 (2q + 1)
    degrees: q = 0 for dx, dy > 0, 1 for dx < 0 < dy, 2 for both negative, 3
    for dy < 0 < dx)."""
    diag = (np.abs(dx) == np.abs(dy)) & (dx != 0)
    q = np.where(dy > 0, np.where(dx > 0, 0, 1), np.where(dx < 0, 2, 3))
    return diag, q


def orientation_vote_margin(L: np.ndarray, xi: int, yi: int, sigma_oct: float, p: Params) -> float:
    """Decision margin of the nearest-bin votes of orientation_histogram (§3.2's
    36-bin histogram): over the same window and samples, the smallest distance,
    in bins, of a voting sample's bin coordinate n * theta / 2 pi from a
    rounding boundary k + 1/2 (where the nearest bin changes). Samples of zero
    weight do not vote, and samples exactly on a boundary (|dx| = |dy|) are
    decided exactly (orientation_histogram), so they are not near one. A vote
    within FP32 rounding of a boundary may land in the neighbouring bin on the
    FP32 path; keypoints with a small margin are the ones whose histogram is
    not a robust function of the image.
    """
    h, w = L.shape
    n = p.ori_bins
    sw = p.ori_sigma_factor * sigma_oct
    R = _round_pos(p.ori_radius_factor * sw)
    j, i = np.meshgrid(np.arange(-R, R + 1), np.arange(-R, R + 1), indexing="ij")
    ys, xs = yi + j, xi + i
    ok = (xs >= 1) & (xs <= w - 2) & (ys >= 1) & (ys <= h - 2)
    ys, xs, i, j = ys[ok], xs[ok], i[ok], j[ok]
    dx, dy = _gradients(L, ys, xs)
    mag = np.sqrt(dx * dx + dy * dy)
    th = np.arctan2(dy, dx)
    th = np.where(th < 0, th + 2 * math.pi, th)
    wt = np.exp(-(i * i + j * j) / (2.0 * sw * sw))
    diag, _ = _diagonal_quadrant(dx, dy)
    votes = (wt * mag > 0) & ~diag
    if not votes.any():
        return math.inf
    t = n * th[votes] / (2 * math.pi) + 0.5   # bin = floor(t) mod n; boundaries at integer t
    f = t - np.floor(t)
    return float(np.minimum(f, 1.0 - f).min())


def smooth_histogram(hist: np.ndarray) -> np.ndarray:
    """One circular pass of [1/4, 1/2, 1/4] (§3.2)."""
    return 0.25 * np.roll(hist, 1) + 0.5 * hist + 0.25 * np.roll(hist, -1)


def orientation_peaks(hist_s: np.ndarray, p: Params):
    """Peaks of the smoothed histogram with parabolic sub-bin refinement (§3.2).

    READING: bin k is a peak when strictly above both circular neighbours and
    >= ori_peak_ratio * max; refined bin k + (h[k-1] - h[k+1]) /
    (2 (h[k-1] - 2 h[k] + h[k+1])); angle = 360 * bin / n in [0, 360).
    Returns (angles in degrees, ascending bin order) and the decision margin
    relative to the histogram maximum.
    """
    n = len(hist_s)
    hmax = float(hist_s.max()) if n else 0.0
    angles = []
    margin = math.inf
    if hmax <= 0:
        return angles, margin
    thr = p.ori_peak_ratio * hmax
    for k in range(n):
        hm, hk, hp = hist_s[(k - 1) % n], hist_s[k], hist_s[(k + 1) % n]
        is_lmax = hk > hm and hk > hp
        above = hk >= thr
        if is_lmax:
            margin = min(margin, abs(hk - thr) / hmax)
        if above or hk >= thr * (1 - 1e-3):
            margin = min(margin, abs(hk - hm) / hmax, abs(hk - hp) / hmax)
        if is_lmax and above:
            kf = k + 0.5 * (hm - hp) / (hm - 2.0 * hk + hp)
            kf = kf % n
            angles.append((360.0 * kf / n) % 360.0)
    return angles, margin


# ------------------------------------------------------------- A8: descriptor

def _trilinear_histogram(u, v, o, wt, p: Params) -> np.ndarray:
    """Accumulate samples at continuous bin coordinates (v, u, o) with weights
    wt into the d x d x nb histogram, each split over its 2 x 2 x 2 nearest
    bins (o circular; spatial bins outside 0..d-1 are dropped)."""
    d, nb = p.desc_width, p.desc_bins
    u0 = np.floor(u).astype(np.int64)
    v0 = np.floor(v).astype(np.int64)
    o0 = np.floor(o).astype(np.int64)
    fu, fv, fo = u - u0, v - v0, o - o0
    hist = np.zeros((d, d, nb))
    for dv in (0, 1):
        wv = fv if dv else 1 - fv
        vv = v0 + dv
        for du in (0, 1):
            wu = fu if du else 1 - fu
            uu = u0 + du
            inb = (vv >= 0) & (vv < d) & (uu >= 0) & (uu < d)
            for do in (0, 1):
                wo = fo if do else 1 - fo
                oo = (o0 + do) % nb
                np.add.at(hist, (vv[inb], uu[inb], oo[inb]), (wt * wv * wu * wo)[inb])
    return hist


def plain_histogram(L: np.ndarray, xk: float, yk: float, xi: int, yi: int, sigma_oct: float,
                    angle_deg: float, p: Params) -> np.ndarray:
    """Raw (unnormalised) 4x4x8 gradient histogram of the single-scale
    descriptor (§3.2), on the pixel grid.

    READING (textbook SIFT): spatial bin width w = desc_scale * sigma; samples are
    the pixels within Chebyshev radius round(w * sqrt(2) * (d + 1) / 2) of the
    integer keypoint pixel; offsets from the sub-pixel keypoint are rotated by
    -theta and divided by w, giving bin coordinates (u, v) = (rx, ry) + d/2 - 1/2,
    kept when -1 < u, v < d; weight m * exp(-(rx^2 + ry^2) / (2 (d/2)^2));
    trilinear split over (v, u, o) with o circular.
    """
    h, w = L.shape
    d, nb = p.desc_width, p.desc_bins
    wbin = p.desc_scale * sigma_oct
    R = _round_pos(wbin * math.sqrt(2.0) * (d + 1) * 0.5)
    th = math.radians(angle_deg)
    ct, st = math.cos(th), math.sin(th)
    j, i = np.meshgrid(np.arange(-R, R + 1), np.arange(-R, R + 1), indexing="ij")
    ys, xs = (yi + j).ravel(), (xi + i).ravel()
    ok = (xs >= 1) & (xs <= w - 2) & (ys >= 1) & (ys <= h - 2)
    ys, xs = ys[ok], xs[ok]
    ox = xs - xk
    oy = ys - yk
    rx = (ct * ox + st * oy) / wbin
    ry = (-st * ox + ct * oy) / wbin
    u = rx + 0.5 * d - 0.5
    v = ry + 0.5 * d - 0.5
    keep = (u > -1) & (u < d) & (v > -1) & (v < d)
    ys, xs, rx, ry, u, v = ys[keep], xs[keep], rx[keep], ry[keep], u[keep], v[keep]
    dx, dy = _gradients(L, ys, xs)
    mag = np.sqrt(dx * dx + dy * dy)
    phi = np.arctan2(dy, dx) - th
    phi = np.mod(phi, 2 * math.pi)
    o = phi * nb / (2 * math.pi)
    wt = mag * np.exp(-(rx * rx + ry * ry) / (2.0 * (0.5 * d) ** 2))
    return _trilinear_histogram(u, v, o, wt, p)


def bilinear(L: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Bilinear interpolation of L at continuous positions (x, y), which must
    satisfy 0 <= x < W - 1 and 0 <= y < H - 1."""
    x0 = np.floor(x).astype(np.int64)
    y0 = np.floor(y).astype(np.int64)
    fx, fy = x - x0, y - y0
    top = (1 - fx) * L[y0, x0] + fx * L[y0, x0 + 1]
    bot = (1 - fx) * L[y0 + 1, x0] + fx * L[y0 + 1, x0 + 1]
    return (1 - fy) * top + fy * bot


def dsp_scale_histogram(L: np.ndarray, xk: float, yk: float, sigma_oct: float,
                        angle_deg: float, scale: float, p: Params) -> np.ndarray:
    """Raw 4x4x8 histogram of one DSP scale (§3.2 "DSP Multi-Scale Descriptor
    Pooling": a 32 x 32 patch per scale).

    READING: the patch is a G x G grid (G = dsp_grid) of samples covering the
    descriptor's d x d spatial bins of width w = desc_scale * sigma * scale,
    G / d samples per bin along each axis, at bin coordinates
    (rx, ry) = ((a + 1/2) d / G - d/2, (b + 1/2) d / G - d/2) from the keypoint
    in its rotated frame; image position (x, y) = (xk, yk) + w R(theta) (rx, ry).
    The gradient there is the central difference of the bilinearly
    interpolated level, dx = L(x+1, y) - L(x-1, y), dy = L(x, y+1) - L(x, y-1);
    samples whose stencil leaves the image (unless 1 <= x < W-2 and
    1 <= y < H-2) are skipped. Weight, orientation bin and the trilinear split
    are those of the single-scale descriptor with (u, v) = (rx, ry) + d/2 - 1/2.
    """
    h, w = L.shape
    d, nb, G = p.desc_width, p.desc_bins, p.dsp_grid
    wbin = p.desc_scale * sigma_oct * scale
    th = math.radians(angle_deg)
    ct, st = math.cos(th), math.sin(th)
    c = (np.arange(G) + 0.5) * d / G - 0.5 * d
    ry, rx = np.meshgrid(c, c, indexing="ij")
    rx, ry = rx.ravel(), ry.ravel()
    x = xk + wbin * (ct * rx - st * ry)
    y = yk + wbin * (st * rx + ct * ry)
    ok = (x >= 1) & (x < w - 2) & (y >= 1) & (y < h - 2)
    x, y, rx, ry = x[ok], y[ok], rx[ok], ry[ok]
    dx = bilinear(L, x + 1, y) - bilinear(L, x - 1, y)
    dy = bilinear(L, x, y + 1) - bilinear(L, x, y - 1)
    mag = np.sqrt(dx * dx + dy * dy)
    phi = np.mod(np.arctan2(dy, dx) - th, 2 * math.pi)
    o = phi * nb / (2 * math.pi)
    wt = mag * np.exp(-(rx * rx + ry * ry) / (2.0 * (0.5 * d) ** 2))
    return _trilinear_histogram(rx + 0.5 * d - 0.5, ry + 0.5 * d - 0.5, o, wt, p)


def normalise_descriptor(hist: np.ndarray, p: Params) -> np.ndarray:
    """L2 normalise, clip at desc_clip, L2 renormalise (zero vector if the
    norm is 0); with rootsift (§3.2 "RootSIFT Normalization"), then divide by
    the L1 norm and take element-wise square roots."""
    vec = hist.ravel().astype(np.float64)
    nrm = math.sqrt(float(vec @ vec))
    if nrm == 0:
        return np.zeros(vec.size)
    vec = np.minimum(vec / nrm, p.desc_clip)
    nrm = math.sqrt(float(vec @ vec))
    vec = vec / nrm if nrm > 0 else vec
    if p.rootsift:
        l1 = float(np.sum(np.abs(vec)))
        vec = np.sqrt(vec / l1) if l1 > 0 else vec
    return vec


def descriptor(L: np.ndarray, xk: float, yk: float, xi: int, yi: int, sigma_oct: float,
               angle_deg: float, p: Params) -> np.ndarray:
    """4x4x8 descriptor (§3.2), layout [v][u][o] row-major: the single-scale
    pixel-grid histogram, or with dsp the mean of the DSP scales' histograms
    (pooled before normalisation, §3.2), then normalise_descriptor."""
    if p.dsp:
        hist = sum(dsp_scale_histogram(L, xk, yk, sigma_oct, angle_deg, f, p)
                   for f in p.dsp_scales) / len(p.dsp_scales)
    else:
        hist = plain_histogram(L, xk, yk, xi, yi, sigma_oct, angle_deg, p)
    return normalise_descriptor(hist, p)


# ------------------------------------------------------------------ A9: cap

def cap_topk(response: np.ndarray, k: int) -> np.ndarray:
    """READING: keep the k largest responses, ties broken by canonical (input)
    order; return the kept indices in canonical order."""
    n = len(response)
    if k <= 0 or n <= k:
        return np.arange(n)
    order = sorted(range(n), key=lambda i: (-response[i], i))
    return np.sort(np.array(order[:k], dtype=np.int64))


# ------------------------------------------------------------------ driver

@dataclass
class Result:
    x: np.ndarray
    y: np.ndarray
    sigma: np.ndarray
    angle: np.ndarray
    response: np.ndarray
    octave: np.ndarray
    layer: np.ndarray
    desc: np.ndarray
    margin: np.ndarray          # smallest decision margin behind each keypoint
    internals: dict = field(default_factory=dict)  # octave-local refinement state per keypoint
    cand: dict = field(default_factory=dict)     # candidate table
    n_refined: int = 0
    pyramid: list = None

    def __len__(self):
        return len(self.x)


def extract(img: np.ndarray, p: Params = None, keep_pyramid: bool = False,
            with_descriptors: bool = True) -> Result:
    """Whole extraction path for one image, stage by stage (§3.2, Eq. 1's
    Pyr -> DoG -> Ext -> Ori -> Desc)."""
    p = p or Params()
    p = for_image(np.shape(img)[0], np.shape(img)[1], p)
    pyr = build_pyramid(img, p)
    scale_up = 0.5 if p.upsample else 1.0
    S = p.n_scales
    rows = []
    cand_tab = {k: [] for k in ("octave", "s", "y", "x", "code", "margin")}
    n_ref = 0
    for o, G in enumerate(pyr):
        D = dog(G)
        cs, cy, cx, mg, me = find_candidates(D, p)
        for ci in range(len(cs)):
            r = refine_candidate(D, int(cs[ci]), int(cy[ci]), int(cx[ci]), p)
            m0 = min(float(mg[ci]), float(me[ci]), r.margin)
            for k, v in (("octave", o), ("s", int(cs[ci])), ("y", int(cy[ci])), ("x", int(cx[ci])),
                         ("code", r.code), ("margin", m0)):
                cand_tab[k].append(v)
            if r.code != KEEP:
                continue
            n_ref += 1
            s_f = r.s + r.ds
            sigma_oct = p.sigma0 * 2.0 ** (s_f / S)
            L = G[r.s]
            if p.upright:
                angles, m1 = [0.0], math.inf
            else:
                hist = orientation_histogram(L, r.x, r.y, sigma_oct, p)
                angles, m1 = orientation_peaks(smooth_histogram(hist), p)
                m1 = min(m1, orientation_vote_margin(L, r.x, r.y, sigma_oct, p))
            for a in angles:
                rows.append((o, r, sigma_oct, a, min(m0, m1)))
    resp = np.array([row[1].response for row in rows])
    keep = cap_topk(resp, p.max_kpts) if p.max_kpts > 0 else np.arange(len(rows))
    n = len(keep)
    out = {k: np.zeros(n) for k in ("x", "y", "sigma", "angle", "response", "margin")}
    octv = np.zeros(n, dtype=np.int64)
    layer = np.zeros(n, dtype=np.int64)
    desc = np.zeros((n, p.desc_width ** 2 * p.desc_bins))
    internals = {k: np.zeros(n) for k in ("xi", "yi", "dx", "dy", "sigma_oct")}
    for t, idx in enumerate(keep):
        o, r, sigma_oct, a, m = rows[idx]
        f = (2.0 ** o) * scale_up
        xk, yk = r.x + r.dx, r.y + r.dy
        out["x"][t] = xk * f
        out["y"][t] = yk * f
        out["sigma"][t] = sigma_oct * f
        out["angle"][t] = a
        out["response"][t] = r.response
        out["margin"][t] = m
        octv[t] = o
        layer[t] = r.s
        for k, v in (("xi", r.x), ("yi", r.y), ("dx", r.dx), ("dy", r.dy), ("sigma_oct", sigma_oct)):
            internals[k][t] = v
        if with_descriptors:
            desc[t] = descriptor(pyr[o][r.s], xk, yk, r.x, r.y, sigma_oct, a, p)
    cand = {k: np.array(v) for k, v in cand_tab.items()}
    return Result(out["x"], out["y"], out["sigma"], out["angle"], out["response"], octv, layer,
                  desc, out["margin"], internals, cand, n_ref, pyr if keep_pyramid else None)
