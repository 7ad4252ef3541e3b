"""Pins for the FP64 oracle: each check compares it with something other than
itself (closed forms, brute force, invariants the mathematics fixes), chosen so
that a dropped term, a wrong sign / index or a transposed operand fails one."""
import math

import numpy as np
import pytest

from oracle import sift_oracle as so
from workloads import synth

RNG = np.random.default_rng(1234)


# ----------------------------------------------------------------- taps / blur

@pytest.mark.parametrize("sigma", [0.8, 1.2263, 1.5199, 2.4525, 3.09])
def test_taps_normalised_symmetric_second_moment(sigma):
    r, w = so.gaussian_taps(sigma)
    assert r == math.ceil(4 * sigma)
    assert len(w) == 2 * r + 1
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_array_equal(w, w[::-1])
    k = np.arange(-r, r + 1)
    var = float((k * k * w).sum())
    # Truncation at 4 sigma can only remove tail variance, and removes < 2e-3 of it.
    assert var <= sigma * sigma * (1 + 1e-12)
    assert (sigma * sigma - var) / (sigma * sigma) < 2e-3
    # Closed form of the sampled, untruncated taps: w_k proportional to exp(-k^2/2s^2).
    np.testing.assert_allclose(w / w[r], np.exp(-(k * k) / (2 * sigma * sigma)), rtol=1e-14)


def _refl(i, n):
    while i < 0 or i >= n:
        i = -i if i < 0 else 2 * (n - 1) - i
    return i


def _brute_blur(img, sigma):
    r, w = so.gaussian_taps(sigma)
    h, wd = img.shape
    out = np.zeros((h, wd))
    for y in range(h):
        for x in range(wd):
            acc = 0.0
            for j in range(-r, r + 1):
                for i in range(-r, r + 1):
                    acc += w[j + r] * w[i + r] * img[_refl(y + j, h), _refl(x + i, wd)]
            out[y, x] = acc
    return out


@pytest.mark.parametrize("shape,sigma", [((7, 9), 1.2), ((16, 13), 1.2263), ((33, 31), 1.5451),
                                         ((20, 24), 3.09)])
def test_separable_blur_equals_bruteforce_2d(shape, sigma):
    r, _ = so.gaussian_taps(sigma)
    if r >= min(shape):
        sigma = (min(shape) - 1) / 4.0 - 0.01
    img = RNG.random(shape)
    np.testing.assert_allclose(so.blur(img, sigma), _brute_blur(img, sigma), atol=1e-12, rtol=0)


def test_pyramid_impulse_variance_bookkeeping():
    """Level i of octave 0 applied total variance sigma_i^2 - sigma_in^2 in each axis."""
    p = so.Params()
    n = 257
    img = np.zeros((n, n))
    img[128, 128] = 1.0
    G = so.build_pyramid(img, p)[0]
    k = np.arange(n) - 128.0
    for i, sig in enumerate(so.level_sigmas(p)):
        lv = G[i]
        mass = lv.sum()
        assert abs(mass - 1.0) < 1e-12
        vx = float((lv.sum(axis=0) * k * k).sum())
        vy = float((lv.sum(axis=1) * k * k).sum())
        target = sig * sig - p.init_blur ** 2
        assert abs(vx - target) / target < 2e-3
        assert abs(vx - vy) < 1e-9


def test_increment_sigmas_closed_form():
    p = so.Params()
    kap = so.increment_sigmas(p)
    # kappa_i = sigma0 * 2^((i-1)/S) * sqrt(2^(2/S) - 1): geometric with ratio 2^(1/S).
    expect = [1.6 * 2 ** ((i - 1) / 3) * math.sqrt(2 ** (2 / 3) - 1) for i in range(1, 6)]
    np.testing.assert_allclose(kap, expect, rtol=1e-14)
    assert [math.ceil(4 * k) for k in kap] == [5, 7, 8, 10, 13]
    assert abs(so.base_sigma(p) - math.sqrt(1.6 ** 2 - 0.25)) < 1e-15
    assert abs(so.base_sigma(so.Params(upsample=True)) - math.sqrt(1.6 ** 2 - 1.0)) < 1e-15


# ------------------------------------------------------------ resampling

def test_upsample_identities():
    img = RNG.random((5, 7))
    u = so.upsample2x(img)
    assert u.shape == (10, 14)
    np.testing.assert_array_equal(u[0::2, 0::2], img)
    np.testing.assert_allclose(u[0::2, 1:-1:2], 0.5 * (img[:, :-1] + img[:, 1:]), rtol=1e-15)
    np.testing.assert_allclose(u[1:-1:2, 0::2], 0.5 * (img[:-1] + img[1:]), rtol=1e-15)
    np.testing.assert_allclose(u[1:-1:2, 1:-1:2],
                               0.25 * (img[:-1, :-1] + img[:-1, 1:] + img[1:, :-1] + img[1:, 1:]),
                               rtol=1e-14)
    np.testing.assert_array_equal(u[-1, 0::2], img[-1])    # clamped last row
    np.testing.assert_array_equal(u[0::2, -1], img[:, -1])  # clamped last column
    np.testing.assert_array_equal(so.decimate(u), img)


@pytest.mark.parametrize("v,want", [
    (1.0 / 3.0, 0.333251953125),            # binary16 0x3555, the nearest to 1/3
    (1.0 + 2.0 ** -11, 1.0),                # halfway between 1 and 1 + 2^-10: ties to even
    (1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -9),  # halfway, the even neighbour is above
    (0.1, 0.0999755859375),                 # binary16 0x2E66
    (2.0 ** -25, 0.0),                      # below half the smallest subnormal 2^-24
    (0.75, 0.75),                           # exactly representable
])
def test_fp16_storage_rounds_to_nearest_binary16(v, want):
    """§3.2's fp16 storage: a stored level of an octave above 0 is the nearest
    IEEE binary16 value, ties to even (values worked out by hand above);
    octave 0 and the default mode keep the value."""
    p16 = so.Params(fp16_pyramid=True)
    a = np.array([[v]])
    assert so.store_level(a, 1, p16)[0, 0] == want
    assert so.store_level(a, 0, p16)[0, 0] == v
    assert so.store_level(a, 3, so.Params())[0, 0] == v


@pytest.mark.parametrize("up", [False, True])
def test_fp16_pyramid_keeps_octave0_and_bounds_the_rest(up):
    """With fp16 storage, octave 0 equals the full-precision pyramid exactly;
    every level above it holds binary16 values; and it differs from the
    full-precision pyramid by at most one half-ulp of [0, 1) values (2^-12)
    per rounding it went through: the taps are non-negative and sum to one,
    so a blur does not grow an earlier error. Level i of octave o has gone
    through (o - 1)(S + 1) + i + 1 roundings."""
    img = synth.make_image(synth.rng_for(10, 7), 150, 190)
    p = so.Params(upsample=up)
    p16 = so.Params(upsample=up, fp16_pyramid=True)
    a, b = so.build_pyramid(img, p), so.build_pyramid(img, p16)
    assert len(a) == len(b) >= 3
    np.testing.assert_array_equal(a[0], b[0])
    S = p.n_scales
    for o in range(1, len(a)):
        assert np.array_equal(b[o].astype(np.float16).astype(np.float64), b[o])
        for i in range(S + 3):
            n_round = (o - 1) * (S + 1) + i + 1
            assert np.abs(b[o][i] - a[o][i]).max() <= n_round * 2.0 ** -12 + 1e-15, (o, i)
    # Octave 1 starts from octave 0's level S, decimated and then rounded once.
    want = so.decimate(a[0][S]).astype(np.float16).astype(np.float64)
    np.testing.assert_array_equal(b[1][0], want)


def test_magnify_limit():
    """§5's suppression of the double image above 4 MP: the limit counts input
    pixels, an image of exactly the limit is still magnified, 0 disables it."""
    p = so.Params(upsample=True, upsample_max_px=1000)
    assert so.magnify(25, 40, p) and so.magnify(40, 25, p)
    assert not so.magnify(25, 41, p) and not so.magnify(41, 25, p)
    d = so.Params(upsample=True)
    assert d.upsample_max_px == 4_000_000
    assert so.magnify(2000, 2000, d) and not so.magnify(2000, 2001, d)
    assert so.octave_sizes(2000, 2000, d)[0] == (4000, 4000)
    assert so.octave_sizes(2000, 2001, d)[0] == (2000, 2001)
    assert so.magnify(5000, 5000, so.Params(upsample=True, upsample_max_px=0))
    assert not so.magnify(10, 10, so.Params(upsample=False, upsample_max_px=0))


def test_suppressed_image_takes_the_plain_path():
    """Above the limit the image is processed exactly as without upsampling
    (octave 0 at the input size, base blur from the unmagnified input, output
    coordinates not halved); at the limit it is magnified."""
    img = RNG.random((40, 52))
    plain = so.extract(img, so.Params())
    supp = so.extract(img, so.Params(upsample=True, upsample_max_px=40 * 52 - 1))
    for k in ("x", "y", "sigma", "angle", "response", "octave", "layer", "desc"):
        np.testing.assert_array_equal(getattr(supp, k), getattr(plain, k))
    assert so.build_pyramid(img, so.Params(upsample=True, upsample_max_px=40 * 52 - 1))[0].shape[1:] == (40, 52)
    assert so.build_pyramid(img, so.Params(upsample=True, upsample_max_px=40 * 52))[0].shape[1:] == (80, 104)


def test_decimate_floor_size_and_octaves():
    img = RNG.random((31, 18))
    d = so.decimate(img)
    assert d.shape == (15, 9)
    np.testing.assert_array_equal(d, img[0:30:2, 0:18:2])
    assert so.octave_sizes(480, 640, so.Params()) == [(480, 640), (240, 320), (120, 160),
                                                        (60, 80), (30, 40)]
    # an octave is kept while its smaller side is at least min_octave_side (16)
    assert so.octave_sizes(16, 16, so.Params()) == [(16, 16)]
    assert so.octave_sizes(32, 40, so.Params()) == [(32, 40), (16, 20)]
    assert so.octave_sizes(15, 100, so.Params()) == []
    assert so.octave_sizes(8, 9, so.Params(upsample=True)) == [(16, 18)]
    assert len(so.octave_sizes(750, 1000, so.Params(upsample=True))) == 7
    assert len(so.octave_sizes(1200, 1600, so.Params(upsample=True))) == 8


# ------------------------------------------------------------------ extrema

def _brute_candidates(D, p):
    S, b = p.n_scales, p.border
    _, h, w = D.shape
    out = []
    for s in range(1, S + 1):
        for y in range(b, h - b):
            for x in range(b, w - b):
                c = D[s, y, x]
                if not abs(c) > p.prefilter_ratio * p.contrast_thr:
                    continue
                nb = [D[s + a, y + bb, x + cc] for a in (-1, 0, 1) for bb in (-1, 0, 1)
                      for cc in (-1, 0, 1) if (a, bb, cc) != (0, 0, 0)]
                if all(c > v for v in nb) or all(c < v for v in nb):
                    out.append((s, y, x))
    return out


def test_extrema_match_bruteforce_loop():
    p = so.Params(contrast_thr=0.02)
    D = RNG.normal(0, 0.02, size=(5, 23, 27))
    D[2, 10, 12] = 0.3    # a planted maximum
    D[1, 15, 7] = -0.3    # a planted minimum
    D[3, 8, 20] = 0.3
    D[3, 8, 21] = 0.3     # a plateau: strictness rejects both
    cs, cy, cx, mg, me = so.find_candidates(D, p)
    got = list(zip(cs.tolist(), cy.tolist(), cx.tolist()))
    want = _brute_candidates(D, p)
    assert got == want
    assert (2, 10, 12) in got and (1, 15, 7) in got
    assert (3, 8, 20) not in got and (3, 8, 21) not in got
    assert np.all(mg > 0) and np.all(me > 0)


def test_quadratic_dog_single_extremum_at_vertex():
    p = so.Params(contrast_thr=0.001)
    s_, y_, x_ = np.mgrid[0:5, 0:21, 0:21].astype(float)
    D = 0.05 - 0.001 * ((x_ - 9) ** 2 + 2 * (y_ - 11) ** 2 + 3 * (s_ - 2) ** 2)
    cs, cy, cx, _, _ = so.find_candidates(D, p)
    assert list(zip(cs, cy, cx)) == [(2, 11, 9)]


# --------------------------------------------------------------- refinement

def _quadratic_stack(vertex, H, c0=0.04, shape=(5, 25, 25)):
    s_, y_, x_ = np.mgrid[0:shape[0], 0:shape[1], 0:shape[2]].astype(float)
    d = np.stack([x_ - vertex[0], y_ - vertex[1], s_ - vertex[2]])
    q = np.einsum("i...,ij,j...->...", d, H, d)
    return c0 + 0.5 * q


def test_cramer_matches_linalg_solve():
    for _ in range(50):
        A = RNG.normal(size=(3, 3))
        A = A @ A.T + 0.1 * np.eye(3)
        bvec = RNG.normal(size=3)
        np.testing.assert_allclose(so.cramer_solve(A, bvec), np.linalg.solve(A, bvec), rtol=1e-9)
    assert so.cramer_solve(np.zeros((3, 3)), np.ones(3)) is None


@pytest.mark.parametrize("off", [(0.3, -0.2, 0.1), (-0.45, 0.4, -0.35), (1.3, -0.2, 0.2),
                                 (-2.2, 1.6, 0.3), (0.55, -0.3, 0.1), (-0.58, 0.52, 0.05)])
def test_refinement_recovers_quadratic_vertex(off):
    """Central differences are exact on a quadratic, so the vertex is recovered
    exactly, after one move per whole-pixel offset; the contrast is the vertex value.
    An offset component of 0.5 or more always moves the pixel (offsets 0.55 and
    -0.58 end at the neighbouring pixel with |offset| < 0.5)."""
    p = so.Params(contrast_thr=0.001)
    H = -np.array([[0.010, 0.002, 0.001], [0.002, 0.012, -0.001], [0.001, -0.001, 0.02]])
    v = (12 + off[0], 12 + off[1], 2 + off[2])
    D = _quadratic_stack(v, H)
    r = so.refine_candidate(D, 2, 12, 12, p)
    assert r.code == so.KEEP
    np.testing.assert_allclose([r.x + r.dx, r.y + r.dy, r.s + r.ds], v, atol=1e-10)
    assert abs(r.response - 0.04) < 1e-12
    assert max(abs(r.dx), abs(r.dy), abs(r.ds)) < 0.5


def test_refinement_rejections():
    p = so.Params(contrast_thr=0.001)
    H = -np.diag([0.01, 0.01, 0.02])
    D = _quadratic_stack((12.2, 12.1, 2.1), H, c0=0.0005)     # low contrast
    assert so.refine_candidate(D, 2, 12, 12, p).code == so.REJ_CONTRAST
    D = _quadratic_stack((12.2, 2.0, 2.1), H, shape=(5, 25, 25))  # vertex outside border
    assert so.refine_candidate(D, 2, 6, 12, p).code == so.REJ_BOUNDS
    D = np.zeros((5, 25, 25))
    assert so.refine_candidate(D, 2, 12, 12, p).code == so.REJ_SINGULAR


@pytest.mark.parametrize("a,b", [(1.0, 1.0), (1.0, 8.0), (1.0, 9.9), (1.0, 10.1), (1.0, 20.0),
                                 (1.0, -1.0)])
def test_edge_test_threshold(a, b):
    """Spatial Hessian diag(a, b) is rejected iff (a+b)^2/(ab) >= (r+1)^2/r or ab <= 0."""
    p = so.Params(contrast_thr=0.001, edge_ratio=10.0)
    H = -0.001 * np.diag([a, b, 5.0])
    D = _quadratic_stack((12.0, 12.0, 2.0), H)
    r = so.refine_candidate(D, 2, 12, 12, p)
    reject = a * b <= 0 or (a + b) ** 2 / (a * b) >= 121.0 / 10.0
    assert (r.code == so.REJ_EDGE) == reject
    if not reject:
        assert r.code == so.KEEP


def _separable_stack(fx, fy, fs, x0, y0, s0, shape=(5, 25, 25), c0=0.0):
    """D = c0 + fx + fy + fs with each profile given on consecutive indices from
    (x0, y0, s0) and zero elsewhere; mixed differences of a separable sum are 0."""
    D = np.full(shape, c0)
    gx, gy, gs = np.zeros(shape[2]), np.zeros(shape[1]), np.zeros(shape[0])
    gx[x0:x0 + len(fx)] = fx
    gy[y0:y0 + len(fy)] = fy
    gs[s0:s0 + len(fs)] = fs
    return D + gs[:, None, None] + gy[None, :, None] + gx[None, None, :]


def test_refinement_half_offset_rounds_away_from_zero():
    """An offset of exactly +-1/2 is not converged (|delta| < 0.5 is required) and
    moves the pixel, rounded half away from zero. A profile 0, 1, 1 along x has
    dx = 1/2 and dxx = -1, so delta_x = 1/2 exactly (powers of two, exact in
    Cramer's rule); at x = W - b - 1 the move lands on the border and is
    rejected, as is the mirrored profile at x = b and the same profile along s
    at the top layer s = S."""
    p = so.Params(contrast_thr=0.001)
    b, S = p.border, p.n_scales
    peak = [0.0, 1.0, 0.0]
    x = 25 - b - 1
    D = _separable_stack([0.0, 1.0, 1.0], peak, peak, x - 1, 11, 1)
    assert so.refine_candidate(D, 2, 12, x, p).code == so.REJ_BOUNDS
    D = _separable_stack([1.0, 1.0, 0.0], peak, peak, b - 1, 11, 1)
    assert so.refine_candidate(D, 2, 12, b, p).code == so.REJ_BOUNDS
    D = _separable_stack(peak, peak, [0.0, 1.0, 1.0], 11, 11, S - 1)
    assert so.refine_candidate(D, S, 12, 12, p).code == so.REJ_BOUNDS


def test_refinement_is_capped_at_five_steps():
    """§3.2 fixes five refinement iterations. Along x the profile f(k+1) =
    (4 f(k) - f(k-1)) / 3 from f = 0, 1 makes every Newton step exactly one
    pixel; ending it with a mirror (f(k+1) = f(k-1)) puts the vertex on a pixel.
    Four moves then converge on the fifth evaluation and are kept; five moves
    exhaust the iterations and are rejected."""
    p = so.Params(contrast_thr=0.001)
    for moves, code in ((4, so.KEEP), (5, so.REJ_NOCONV)):
        f = [0.0, 1.0]
        for _ in range(moves):
            f.append((4 * f[-1] - f[-2]) / 3)
        f.append(f[-2])
        peak = [-1 / 81, 0.0, -1 / 81]
        D = _separable_stack(f, peak, [-2 / 81, 0.0, -2 / 81], 7, 11, 1)
        r = so.refine_candidate(D, 2, 12, 8, p)
        assert r.code == code, moves
        if code == so.KEEP:
            assert r.x == 8 + moves and abs(r.dx) < 1e-9


def test_edge_ratio_at_exact_threshold_is_rejected():
    """Principal curvatures in ratio exactly r = 10 (dxx = -10, dyy = -1, all
    integers) give tr^2 r = (r + 1)^2 det = 1210; only tr^2 r < (r + 1)^2 det
    passes, so the candidate is rejected as an edge."""
    p = so.Params(contrast_thr=0.001, edge_ratio=10.0)
    D = _separable_stack([-5.0, 0.0, -5.0], [-0.5, 0.0, -0.5], [-0.5, 0.0, -0.5], 11, 11, 1,
                         c0=20.0)
    assert so.refine_candidate(D, 2, 12, 12, p).code == so.REJ_EDGE
    D = _separable_stack([-5.0, 0.0, -5.0], [-0.5625, 0.0, -0.5625], [-0.5, 0.0, -0.5],
                         11, 11, 1, c0=20.0)   # ratio 10 / 1.125: kept
    assert so.refine_candidate(D, 2, 12, 12, p).code == so.KEEP


def test_refinement_margin_reports_the_convergence_decision():
    """The margin is the smallest relative distance of any decision from its
    threshold: a vertex 0.45 px off converges with |0.5 - 0.45| / 0.5 = 0.1,
    nearer than the contrast and edge decisions here."""
    p = so.Params(contrast_thr=0.001)
    H = -np.diag([0.01, 0.012, 0.02])
    D = _quadratic_stack((12.45, 12.1, 2.1), H)
    r = so.refine_candidate(D, 2, 12, 12, p)
    assert r.code == so.KEEP
    assert abs(r.margin - 0.1) < 1e-9


def test_candidate_margins_are_relative_distances():
    """Each candidate carries two margins: the pre-gate's (|D| - T') / max(|D|, T')
    with T' = contrast_thr / 2, and the extremum's gap to the nearest of its 26
    neighbours relative to |D|. A maximum 0.1 beside 0.08 has gap 0.2; a minimum
    -0.1 beside -0.05 has gap 0.5."""
    p = so.Params()
    D = np.zeros((5, 21, 21))
    D[2, 7, 7], D[2, 7, 8] = 0.1, 0.08
    D[3, 12, 12], D[3, 12, 13] = -0.1, -0.05
    cs, cy, cx, mg, me = so.find_candidates(D, p)
    assert list(zip(cs, cy, cx)) == [(2, 7, 7), (3, 12, 12)]
    gate = 0.5 * p.contrast_thr
    np.testing.assert_allclose(mg, [(0.1 - gate) / 0.1] * 2, rtol=1e-12)
    np.testing.assert_allclose(me, [0.2, 0.5], rtol=1e-12)


@pytest.mark.parametrize("vertex,c0,diag,want", [
    ((13.3, 12.1, 2.1), 0.04, (10.0, 12.0, 20.0), 0.2 / 1.5),   # move of 1.3: 0.2 from the 1.5 rounding edge
    ((12.1, 12.1, 2.1), 0.0011, (10.0, 12.0, 20.0), 0.0001 / 0.0011),   # contrast 0.0011 vs 0.001
    ((12.1, 12.1, 2.1), 0.04, (1.0, 9.0, 5.0), 89.0 / 2089.0),   # edge: |121*9 - 10*10^2| / (1089 + 1000)
])
def test_refinement_margin_takes_the_nearest_decision(vertex, c0, diag, want):
    """The refinement margin is the smallest of: |0.5 - max|delta|| / 0.5 per
    step, |a - (floor(a) + 1/2)| / (floor(a) + 1/2) per moved offset component a,
    the contrast's | |c| - T| / max(|c|, T), and the edge test's
    |(r+1)^2 det - r tr^2| / (|r tr^2| + |(r+1)^2 det|). Each case makes one of the
    last three the smallest."""
    p = so.Params(contrast_thr=0.001)
    H = -1e-3 * np.diag(diag)
    D = _quadratic_stack(vertex, H, c0=c0)
    r = so.refine_candidate(D, 2, 12, 12, p)
    assert r.code == so.KEEP
    assert abs(r.margin - want) < 1e-9


def test_refinement_of_a_minimum_reports_positive_response():
    """The response is |D| at the refined position: a minimum with value -0.04
    reports 0.04."""
    p = so.Params(contrast_thr=0.001)
    H = np.diag([0.010, 0.012, 0.02])
    D = _quadratic_stack((12.2, 11.9, 2.1), H, c0=-0.04)
    r = so.refine_candidate(D, 2, 12, 12, p)
    assert r.code == so.KEEP and abs(r.response - 0.04) < 1e-12


def test_orientation_peak_margins():
    """The peak margin is the distance of every local maximum from the 0.8 ratio
    and, for bins at or near it, of the gap to each neighbour, both relative to
    the maximum: a secondary maximum at 0.75 gives 0.05; a shoulder at 0.99 beside
    the maximum gives 0.01."""
    h = np.zeros(36)
    h[5], h[20] = 1.0, 0.75
    angles, m = so.orientation_peaks(h, so.Params())
    assert angles == [50.0] and abs(m - 0.05) < 1e-12
    h[20], h[6] = 0.0, 0.99
    _, m = so.orientation_peaks(h, so.Params())
    assert abs(m - 0.01) < 1e-12


def test_extract_cap_keeps_the_largest_responses_in_canonical_order():
    """With max_kpts = k the output is the k keypoints of largest response out
    of the uncapped output (equal responses, e.g. the orientations of one point,
    in canonical order), in the same canonical order."""
    img = synth.make_image(synth.rng_for(93, 0), 96, 120)
    full = so.extract(img, so.Params(), with_descriptors=False)
    assert len(full) >= 6
    for k in (1, 2, 3, len(full) - 1):
        cap = so.extract(img, so.Params(max_kpts=k), with_descriptors=False)
        top = np.sort(np.argsort(-full.response, kind="stable")[:k])
        np.testing.assert_array_equal(cap.x, full.x[top])
        np.testing.assert_array_equal(cap.response, full.response[top])


def test_upright_gives_one_keypoint_at_angle_zero_per_refined_point():
    """Upright mode skips the orientation histogram: every refined point gives
    exactly one keypoint, at angle 0."""
    img = synth.make_image(synth.rng_for(93, 0), 96, 120)
    res = so.extract(img, so.Params(upright=True), with_descriptors=False)
    assert len(res) == res.n_refined and len(res) > 0
    assert np.all(res.angle == 0.0)


def test_keypoint_margin_is_the_minimum_over_its_decisions(monkeypatch):
    """A keypoint's margin is the smallest margin of every decision behind it:
    pre-gate, extremum, refinement, orientation peaks and orientation votes.
    Making each stage's
    margin tiny in turn (by wrapping the stage) must bring every keypoint's
    margin down to it."""
    img = synth.make_image(synth.rng_for(93, 0), 96, 120)
    p = so.Params()
    base = so.extract(img, p, with_descriptors=False)
    assert len(base) >= 5 and base.margin.min() > 1e-6
    fc, op = so.find_candidates, so.orientation_peaks

    def cand_stage(k, v):
        def f(D, pp):
            out = list(fc(D, pp))
            out[k] = np.full(len(out[k]), v)
            return tuple(out)
        return f

    for k, v in ((3, 1e-9), (4, 2e-9)):
        monkeypatch.setattr(so, "find_candidates", cand_stage(k, v))
        res = so.extract(img, p, with_descriptors=False)
        assert len(res) == len(base) and np.all(res.margin == v), k
    monkeypatch.setattr(so, "find_candidates", fc)
    monkeypatch.setattr(so, "orientation_peaks", lambda hs, pp: (op(hs, pp)[0], 3e-9))
    res = so.extract(img, p, with_descriptors=False)
    assert len(res) == len(base) and np.all(res.margin == 3e-9)
    monkeypatch.setattr(so, "orientation_peaks", op)
    monkeypatch.setattr(so, "orientation_vote_margin", lambda *a: 4e-9)
    res = so.extract(img, p, with_descriptors=False)
    assert len(res) == len(base) and np.all(res.margin == 4e-9)


def test_dog_is_next_level_minus_this_one():
    """§3.2: D_i = G_{i+1} - G_i. Each further blur lowers the centre of a bright
    blob and raises the centre of a dark one, so D is negative at the first and
    positive at the second, on every layer of every octave."""
    n = 64
    Y, X = np.mgrid[0:n, 0:n].astype(float)
    blob = np.exp(-((X - 31.5) ** 2 + (Y - 31.5) ** 2) / (2 * 3.0 ** 2))
    p = so.Params(min_octave_side=16)
    for sign in (1.0, -1.0):
        for G in so.build_pyramid(0.5 + 0.4 * sign * blob, p):
            D = so.dog(G)
            c = D.shape[1] // 2
            centre = D[:, c - 1:c + 1, c - 1:c + 1].mean(axis=(1, 2))
            assert np.all(-sign * centre > 0), (sign, centre)


# ------------------------------------------------------------------ blob scale

@pytest.mark.parametrize("s", [3.0, 4.0, 6.0, 8.0, 11.0, 16.0])
def test_blob_detected_at_predicted_scale(s):
    """Continuous DoG of a Gaussian blob of width s between sigma and k*sigma peaks
    at sigma* = sqrt(s^2 - sigma_in^2) / sqrt(k); the blob centre has dx = dy = 0."""
    p = so.Params(contrast_thr=0.001)
    n = 257 if s < 10 else 513
    c = n // 2
    Y, X = np.mgrid[0:n, 0:n]
    img = 0.5 + 0.3 * np.exp(-((X - c) ** 2 + (Y - c) ** 2) / (2 * s * s))
    r = so.extract(img, p, with_descriptors=False)
    sel = (np.abs(r.x - c) < 1) & (np.abs(r.y - c) < 1)
    assert sel.any()
    pred = math.sqrt(s * s - p.init_blur ** 2) / math.sqrt(2 ** (1 / 3))
    assert np.all(np.abs(r.sigma[sel] - pred) / pred < 1e-2)
    assert np.all(np.abs(r.x[sel] - c) < 1e-9) and np.all(np.abs(r.y[sel] - c) < 1e-9)


# ------------------------------------------------------------------ orientation

@pytest.mark.parametrize("deg,want_bin", [(45.0, 5), (135.0, 14), (225.0, 23), (315.0, 32)])
def test_diagonal_gradient_votes_upward(deg, want_bin):
    """A gradient with |dx| = |dy| sits exactly on a bin boundary (36 theta / 360
    = 4.5, 13.5, 22.5, 31.5); the nearest-bin rule floor(c + 1/2) sends it to
    the upper bin, 5, 14, 23 or 32. Such samples are decided exactly, so they
    do not count as near a boundary in the vote margin."""
    p = so.Params()
    c, s = round(math.cos(math.radians(deg))), round(math.sin(math.radians(deg)))
    Y, X = np.mgrid[0:61, 0:61].astype(float)
    L = 0.01 * (c * X + s * Y)
    hist = so.orientation_histogram(L, 30, 30, 2.0, p)
    assert list(np.nonzero(hist)[0]) == [want_bin]
    assert so.orientation_vote_margin(L, 30, 30, 2.0, p) == math.inf


@pytest.mark.parametrize("deg", [0.0, 30.0, 90.0, 200.0, 313.0, 47.0])
def test_ramp_orientation(deg):
    """A linear ramp has the same gradient everywhere: its orientation is the
    nearest bin centre, exactly (the smoothed peak is symmetric)."""
    p = so.Params()
    th = math.radians(deg)
    Y, X = np.mgrid[0:101, 0:101].astype(float)
    L = 0.01 * (math.cos(th) * X + math.sin(th) * Y)
    hist = so.orientation_histogram(L, 50, 50, 2.0, p)
    nz = np.nonzero(hist)[0]
    assert len(nz) == 1 and nz[0] == int(math.floor(deg / 10 + 0.5)) % 36
    angles, _ = so.orientation_peaks(so.smooth_histogram(hist), p)
    assert len(angles) == 1
    assert abs(angles[0] - 10 * (int(math.floor(deg / 10 + 0.5)) % 36)) < 1e-9


@pytest.mark.parametrize("deg,want", [(5.0, 0.0), (15.0, 0.0), (355.0, 0.0), (10.0, 0.5),
                                      (7.5, 0.25), (2.5, 0.25), (181.0, 0.4)])
def test_orientation_vote_margin_on_ramps(deg, want):
    """The nearest-bin vote of a sample changes at bin coordinates k + 1/2, i.e.
    at angles 5 + 10 k degrees. A ramp gives every sample the same angle, so the
    vote margin is that angle's distance from the nearest such boundary, in
    bins: 0 on a boundary (5, 15 and 355 degrees, the last one next to the wrap
    at 360), 1/2 at a bin centre, 1/4 a quarter bin off a centre, 0.4 at 181
    degrees (0.1 bin past the centre 180). Float rounding of the angle moves
    these by far less than 1e-9 bins."""
    p = so.Params()
    th = math.radians(deg)
    Y, X = np.mgrid[0:101, 0:101].astype(float)
    L = 0.01 * (math.cos(th) * X + math.sin(th) * Y)
    m = so.orientation_vote_margin(L, 50, 50, 2.0, p)
    assert abs(m - want) < 1e-9


def test_orientation_vote_margin_is_the_minimum_over_voting_samples():
    """One pixel of a ramp at a bin centre (margin 1/2) is changed so that its
    gradient sits 0.01 bin from a boundary: the window's margin becomes 0.01;
    outside the window, or in the ignored outer ring of the image, it does not
    count."""
    p = so.Params()
    Y, X = np.mgrid[0:101, 0:101].astype(float)
    L = 0.01 * X                       # gradient angle 0: a bin centre
    assert abs(so.orientation_vote_margin(L, 50, 50, 2.0, p) - 0.5) < 1e-12
    # Sample (53, 50): dx = L[50, 54] - L[50, 52] = 0.02, dy = L[51, 53] - L[49, 53].
    # Angle (5 - 0.1) degrees, 0.01 bin below the boundary between bins 0 and 1.
    t = math.radians(4.9)
    L2 = L.copy()
    L2[51, 53] = L[51, 53] + 0.5 * 0.02 * math.tan(t)
    L2[49, 53] = L[49, 53] - 0.5 * 0.02 * math.tan(t)
    assert abs(so.orientation_vote_margin(L2, 50, 50, 2.0, p) - 0.01) < 1e-9
    R = int(math.floor(3.0 * 1.5 * 2.0 + 0.5))   # window radius 9
    assert abs(so.orientation_vote_margin(L2, 50 - R - 4, 50, 2.0, p) - 0.5) < 1e-12
    # A flat window casts no vote: no vote decision, no margin.
    assert so.orientation_vote_margin(np.full((40, 40), 0.5), 20, 20, 2.0, p) == math.inf


def test_smoothing_and_parabola():
    h = np.zeros(36)
    h[5] = 4.0
    np.testing.assert_allclose(so.smooth_histogram(h)[[4, 5, 6]], [1.0, 2.0, 1.0])
    assert so.smooth_histogram(h).sum() == pytest.approx(4.0)
    # A parabola sampled at integer bins: refinement returns its exact vertex.
    k = np.arange(36)
    k0 = 17.3
    hp = np.maximum(10.0 - (k - k0) ** 2, 0.0)
    angles, _ = so.orientation_peaks(hp, so.Params())
    assert len(angles) == 1 and abs(angles[0] - 10 * k0) < 1e-9
    # Circular wrap: vertex at -0.2 reports 358 degrees.
    hp = np.maximum(10.0 - ((k + 18) % 36 - 18 + 0.2) ** 2, 0.0)
    angles, _ = so.orientation_peaks(hp, so.Params())
    assert len(angles) == 1 and abs(angles[0] - 358.0) < 1e-9


@pytest.mark.parametrize("ratio,npeaks", [(0.85, 2), (0.79, 1)])
def test_secondary_peak_ratio(ratio, npeaks):
    h = np.zeros(36)
    h[3], h[20] = 1.0, ratio
    angles, _ = so.orientation_peaks(h, so.Params())
    assert len(angles) == npeaks
    assert abs(angles[0] - 30.0) < 1e-9


# ------------------------------------------------------------------ descriptor

def test_descriptor_uniform_gradient_upright_two_bins():
    """Upright on a uniform gradient at angle a: mass only in the two orientation
    bins bracketing a*8/360; exactly one bin when a is a bin centre."""
    p = so.Params()
    Y, X = np.mgrid[0:121, 0:121].astype(float)
    for deg, bins in ((100.0, {2, 3}), (45.0, {1}), (270.0, {6})):
        th = math.radians(deg)
        L = 0.01 * (math.cos(th) * X + math.sin(th) * Y)
        d = so.descriptor(L, 60.3, 59.8, 60, 60, 2.5, 0.0, p).reshape(4, 4, 8)
        assert abs(np.linalg.norm(d) - 1.0) < 1e-12
        nz = set(np.nonzero(d.sum(axis=(0, 1)) > 1e-9)[0].tolist())
        assert nz == bins


def test_descriptor_clip_and_norm():
    p = so.Params()
    L = RNG.random((80, 80))
    d = so.descriptor(L, 40.2, 39.7, 40, 40, 2.2, 37.0, p)
    assert abs(np.linalg.norm(d) - 1.0) < 1e-12
    assert np.all(d >= 0)
    # Before the final renormalisation no entry exceeds the clip: after it, the
    # largest entry is at most clip / ||clipped||.
    assert d.max() <= 0.2 / np.linalg.norm(np.minimum(d, 0.2)) + 1e-12
    assert np.all(so.descriptor(np.zeros((40, 40)), 20, 20, 20, 20, 2.0, 0.0, p) == 0)


# ------------------------------------------------------------------ equivariance

def _match_sets(a_keys, b_keys, tol):
    a = np.asarray(a_keys)
    b = np.asarray(b_keys)
    used = np.zeros(len(b), bool)
    pairs = []
    for i in range(len(a)):
        d = np.abs(b - a[i]).max(axis=1)
        d[used] = np.inf
        j = int(np.argmin(d))
        if d[j] < tol:
            used[j] = True
            pairs.append((i, j))
    return pairs


def _angle_diff(a, b):
    return np.abs((a - b + 180.0) % 360.0 - 180.0)


@pytest.mark.parametrize("dsp", [False, True])
def test_rot90_equivariance_octave0(dsp):
    """Under a 90-degree counter-clockwise rotation (x, y) -> (y, W-1-x), octave-0
    keypoints map one to one, the orientation shifts by -90 degrees and the
    descriptor is unchanged (octave 0 involves no decimation, so it commutes).
    The DSP sample grids are symmetric about the keypoint, so they rotate onto
    themselves and the pooled descriptor is unchanged too."""
    p = so.Params(dsp=dsp)
    img = synth.make_image(synth.rng_for(90, 0), 96, 112)
    r0 = so.extract(img, p)
    r1 = so.extract(np.rot90(img).copy(), p)
    w = img.shape[1]
    m0 = r0.octave == 0
    m1 = r1.octave == 0
    assert m0.sum() == m1.sum() and m0.sum() > 5
    k0 = np.stack([r0.y[m0], w - 1 - r0.x[m0]], 1)
    k1 = np.stack([r1.x[m1], r1.y[m1]], 1)
    a0 = (r0.angle[m0] - 90.0) % 360.0
    a1 = r1.angle[m1]
    pairs = _match_sets(np.c_[k0, a0 / 1e3], np.c_[k1, a1 / 1e3], 1e-6)
    assert len(pairs) == m0.sum()
    d0 = r0.desc[m0]
    d1 = r1.desc[m1]
    for i, j in pairs:
        assert _angle_diff(a0[i], a1[j]) < 1e-6
        np.testing.assert_allclose(d0[i], d1[j], atol=1e-9)


@pytest.mark.parametrize("dsp", [False, True])
def test_rot90_upright_descriptor_permutation(dsp):
    """Upright mode: rotating the image permutes the descriptor as
    (v, u, o) -> (3 - u, v, o - 2 mod 8)."""
    p = so.Params(upright=True, dsp=dsp)
    img = synth.make_image(synth.rng_for(90, 1), 96, 96)
    r0 = so.extract(img, p)
    r1 = so.extract(np.rot90(img).copy(), p)
    w = img.shape[1]
    m0, m1 = r0.octave == 0, r1.octave == 0
    k0 = np.stack([r0.y[m0], w - 1 - r0.x[m0]], 1)
    k1 = np.stack([r1.x[m1], r1.y[m1]], 1)
    pairs = _match_sets(k0, k1, 1e-6)
    assert len(pairs) == m0.sum() == m1.sum() > 3
    d0 = r0.desc[m0].reshape(-1, 4, 4, 8)
    d1 = r1.desc[m1].reshape(-1, 4, 4, 8)
    for i, j in pairs:
        want = np.empty((4, 4, 8))
        for v in range(4):
            for u in range(4):
                for o in range(8):
                    want[3 - u, v, (o - 2) % 8] = d0[i, v, u, o]
        np.testing.assert_allclose(d1[j], want, atol=1e-9)


@pytest.mark.parametrize("dsp", [False, True])
def test_transpose_equivariance_all_octaves(dsp):
    """Transposing the image commutes with blur, decimation and upsampling, so every
    keypoint maps (x, y) -> (y, x) with angle 90 - a, and the descriptor mirrors:
    (v, u, o) -> (3 - v, u, -o mod 8)."""
    p = so.Params(upsample=True, dsp=dsp)
    img = synth.make_image(synth.rng_for(91, 0), 70, 90)
    r0 = so.extract(img, p)
    r1 = so.extract(img.T.copy(), p)
    assert len(r0) == len(r1) > 10
    assert set(r0.octave.tolist()) == set(r1.octave.tolist()) and r0.octave.max() >= 2
    a0 = (90.0 - r0.angle) % 360.0
    k0 = np.c_[r0.y, r0.x, r0.sigma, a0 / 1e3]
    k1 = np.c_[r1.x, r1.y, r1.sigma, r1.angle / 1e3]
    pairs = _match_sets(k0, k1, 1e-6)
    assert len(pairs) == len(r0)
    d0 = r0.desc.reshape(-1, 4, 4, 8)
    d1 = r1.desc.reshape(-1, 4, 4, 8)
    for i, j in pairs:
        want = np.empty((4, 4, 8))
        for v in range(4):
            for u in range(4):
                for o in range(8):
                    want[3 - v, u, (-o) % 8] = d0[i, v, u, o]
        np.testing.assert_allclose(d1[j], want, atol=1e-9)


# ------------------------------------------------------------- DSP / RootSIFT

def test_bilinear_reproduces_bilinear_functions():
    """Bilinear interpolation is exact on f = a + bx + cy + exy and returns the
    sample itself at integer nodes."""
    Y, X = np.mgrid[0:20, 0:30].astype(float)
    a, b, c, e = 0.3, -0.02, 0.05, 0.001
    L = a + b * X + c * Y + e * X * Y
    x = RNG.uniform(0, 28.999, 200)
    y = RNG.uniform(0, 18.999, 200)
    np.testing.assert_allclose(so.bilinear(L, x, y), a + b * x + c * y + e * x * y, atol=1e-12)
    xi = RNG.integers(0, 29, 50).astype(float)
    yi = RNG.integers(0, 19, 50).astype(float)
    np.testing.assert_array_equal(so.bilinear(L, xi, yi), L[yi.astype(int), xi.astype(int)])


@pytest.mark.parametrize("deg", [0.0, 45.0, 120.0])
def test_dsp_ramp_is_scale_invariant_and_separable(deg):
    """On a linear ramp every sample's gradient is the same vector (bilinear
    interpolation is exact on it), and each DSP scale samples the same pattern
    in bin units, so every scale gives the same normalised histogram and the
    pooled descriptor equals any single scale's. Its spatial mass is the outer
    product of one symmetric profile with itself, all in the two orientation
    bins bracketing the gradient angle (one bin at a bin centre)."""
    p = so.Params(dsp=True)
    Y, X = np.mgrid[0:200, 0:200].astype(float)
    th = math.radians(deg)
    L = 0.004 * (math.cos(th) * X + math.sin(th) * Y)
    xk, yk, sig = 100.25, 99.6, 1.9
    pooled = so.descriptor(L, xk, yk, 100, 100, sig, 0.0, p)
    for f in p.dsp_scales:
        one = so.normalise_descriptor(so.dsp_scale_histogram(L, xk, yk, sig, 0.0, f, p), p)
        np.testing.assert_allclose(one, pooled, atol=1e-12)
    h = so.dsp_scale_histogram(L, xk, yk, sig, 0.0, 1.0, p)
    ob = set(np.nonzero(h.sum(axis=(0, 1)) > 1e-12)[0].tolist())
    k = deg * 8 / 360.0
    assert ob == ({int(k)} if k == int(k) else {int(k), int(k) + 1})
    sp = h.sum(axis=2)
    assert np.linalg.matrix_rank(sp, tol=1e-9 * sp.max()) == 1
    np.testing.assert_allclose(sp, sp.T, rtol=1e-12)
    np.testing.assert_allclose(sp, sp[::-1, ::-1], rtol=1e-12)


def test_dsp_patch_mass_closed_form():
    """On L = x/2 (gradient (1, 0): magnitude 1, all mass in orientation bin 0)
    each DSP scale's histogram mass is a closed form of the G x G patch: the
    Gaussian weight and the trilinear split are separable, so the total is
    (sum_a g(c_a) k(u_a))^2 over the G sample coordinates c_a = (a + 1/2) d/G
    - d/2, with g(c) = exp(-c^2 / 8), u = c + 3/2 and k(u) the share of a
    sample's split that stays inside bins 0..3 (1 + u below 0, 4 - u above 3).
    A wrong grid offset, spacing, patch size or weight width changes it."""
    p = so.Params(dsp=True)
    Y, X = np.mgrid[0:300, 0:300].astype(float)
    L = 0.5 * X
    c = (np.arange(p.dsp_grid) + 0.5) * 4 / p.dsp_grid - 2.0
    u = c + 1.5
    k = np.where(u < 0, 1 + u, np.where(u > 3, 4 - u, 1.0))
    want = (np.exp(-c * c / 8.0) * k).sum() ** 2
    for f in p.dsp_scales:
        h = so.dsp_scale_histogram(L, 150.0, 150.0, 2.0, 0.0, f, p)
        assert h[:, :, 1:].sum() == 0.0
        assert h.sum() == pytest.approx(want, rel=1e-12)


def test_dsp_patch_extent_per_scale():
    """Scale f's patch spans d * w_f = 4 * 3 * sigma * f pixels; with sigma = 2 and
    upright sampling its samples lie within (2 - 1/16) * 6 f = 11.625 f px of the
    keypoint. A step edge between columns 70 and 71 changes the interpolated
    level only for x > 70, i.e. for samples more than 9 px right of a keypoint at
    x = 60 (the stencil reaches x + 1): scales 0.5 and 1/sqrt(2) (reach 5.8 and
    8.2 px) see nothing, scales 1, sqrt(2) and 2 (11.6 to 23.3 px) see it."""
    p = so.Params(dsp=True)
    L = np.zeros((120, 120))
    L[:, 71:] = 1.0
    for f in p.dsp_scales:
        h = so.dsp_scale_histogram(L, 60.0, 60.0, 2.0, 0.0, f, p)
        if f < 0.8:
            assert h.sum() == 0.0, f
        else:
            assert h.sum() > 0.0, f


def test_dsp_pooled_scale_mean_on_quadratic():
    """On L = x^2 the central difference of the bilinear level is exactly 4x
    (the interpolation error f(1 - f) is the same at x + 1 and x - 1) and
    dy = 0, so every sample votes 4 (xk + w_f rx) into orientation bin 0.
    Scale f's histogram column u is then 4 (xk A_u + w_f B_u) with A, B fixed
    sums over the bin-unit grid; A is mirror-symmetric and B antisymmetric,
    so the outer columns' ratio r gives (r - 1)/(r + 1) = w B_3 / (xk A_3), with
    w the mean bin width over the pooled scales. Against a single scale f = 1 it
    must be the mean of the five relative scales of §3.2 (1/2 to 2 in steps
    of sqrt 2)."""
    Y, X = np.mgrid[0:128, 0:128].astype(float)
    L = X * X
    xk, yk, sig = 64.3, 63.7, 2.0

    def t(p):
        D = so.descriptor(L, xk, yk, 64, 64, sig, 0.0, p).reshape(4, 4, 8)
        assert D[:, :, 1:].sum() < 1e-12 * D.sum()   # dy rounds to about 1e-13
        col = D.sum(axis=(0, 2))
        r = col[3] / col[0]
        return (r - 1) / (r + 1)

    five = (0.5, 2 ** -0.5, 1.0, 2 ** 0.5, 2.0)
    pooled = t(so.Params(dsp=True, desc_clip=1.0))
    single = t(so.Params(dsp=True, desc_clip=1.0, dsp_scales=(1.0,)))
    assert pooled / single == pytest.approx(sum(five) / 5, rel=1e-9)


@pytest.mark.parametrize("side", ["left", "right", "top", "bottom"])
def test_dsp_stencil_bound_at_image_edge(side):
    """A DSP sample is kept only if its stencil stays inside: 1 <= x < W - 2
    and 1 <= y < H - 2 (the bilinear read at x + 1 needs x + 1 < W - 1). With
    sigma = 2 and scale 2 the bin width is 12 px and the outermost sample
    coordinate is 1.9375 bins, 23.25 px from the keypoint; a keypoint 23.25 px
    inside the edge puts one row (or column) of 32 samples exactly on the
    bound: kept at x = 1 (y = 1), dropped at x = W - 2 (y = H - 2). On a unit
    gradient the mass is the separable closed form of the patch with that
    row or column's share removed when it is dropped."""
    p = so.Params(dsp=True)
    H, W = 160, 150
    Y, X = np.mgrid[0:H, 0:W].astype(float)
    L = 0.5 * (Y if side in ("top", "bottom") else X)
    xk, yk = {"left": (1 + 23.25, 80.0), "right": (W - 2 - 23.25, 80.0),
              "top": (75.0, 1 + 23.25), "bottom": (75.0, H - 2 - 23.25)}[side]
    c = (np.arange(p.dsp_grid) + 0.5) * 4 / p.dsp_grid - 2.0
    u = c + 1.5
    k = np.where(u < 0, 1 + u, np.where(u > 3, 4 - u, 1.0)) * np.exp(-c * c / 8.0)
    full = k.sum()
    edge = full - k[-1] if side in ("right", "bottom") else full
    h = so.dsp_scale_histogram(L, xk, yk, 2.0, 0.0, 2.0, p)
    assert h.sum() == pytest.approx(edge * full, rel=1e-12)


def test_rootsift_is_sqrt_of_l1_normalised_plain():
    """RootSIFT output squared equals the plain (clipped, L2-renormalised)
    descriptor divided by its L1 norm; it has unit L2 norm and no negative entry."""
    img = synth.make_image(synth.rng_for(92, 0), 90, 110)
    r0 = so.extract(img, so.Params())
    r1 = so.extract(img, so.Params(rootsift=True))
    assert len(r0) == len(r1) > 5
    l1 = r0.desc.sum(axis=1, keepdims=True)
    np.testing.assert_allclose(r1.desc ** 2, r0.desc / l1, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(r1.desc, axis=1), 1.0, atol=1e-12)
    assert np.all(r1.desc >= 0)


# ------------------------------------------------------------------ cap

def test_cap_topk_bruteforce():
    resp = RNG.integers(0, 20, size=200).astype(float)  # many ties
    for k in (0, 1, 7, 50, 199, 200, 300):
        got = so.cap_topk(resp, k)
        if k <= 0 or k >= len(resp):
            np.testing.assert_array_equal(got, np.arange(len(resp)))
            continue
        # Brute force: keep i iff fewer than k elements precede it in (-resp, index) order.
        keep = [i for i in range(len(resp))
                if sum(1 for j in range(len(resp))
                       if (resp[j] > resp[i]) or (resp[j] == resp[i] and j < i)) < k]
        np.testing.assert_array_equal(got, keep)


def test_refinement_move_onto_border_is_rejected():
    """A move that lands on x = W - b leaves the band [b, W - b) and is rejected;
    one that lands on x = W - b - 1 is kept."""
    p = so.Params(contrast_thr=0.001)
    H = -np.diag([0.01, 0.012, 0.02])
    w = 25
    b = p.border
    D = _quadratic_stack((w - b - 1 + 0.2, 12.0, 2.0), H)   # one move right, stays inside
    r = so.refine_candidate(D, 2, 12, w - b - 2, p)
    assert r.code == so.KEEP and r.x == w - b - 1
    D = _quadratic_stack((w - b + 0.2, 12.0, 2.0), H)       # one move right, onto the edge
    assert so.refine_candidate(D, 2, 12, w - b - 1, p).code == so.REJ_BOUNDS
    D = _quadratic_stack((b - 1 + 0.1, 12.0, 2.0), H)       # one move left, onto b - 1
    assert so.refine_candidate(D, 2, 12, b, p).code == so.REJ_BOUNDS


@pytest.mark.parametrize("sigma_oct", [1.8, 2.5, 3.4])
def test_orientation_window_mass_closed_form(sigma_oct):
    """On a ramp every sample has the same magnitude, so the histogram's total is
    m * (sum_k exp(-k^2 / (2 (1.5 sigma)^2)))^2 over k = -R..R, R = round(4.5 sigma)."""
    p = so.Params()
    Y, X = np.mgrid[0:121, 0:121].astype(float)
    L = 0.003 * X + 0.004 * Y
    m = 2.0 * math.hypot(0.003, 0.004)
    hist = so.orientation_histogram(L, 60, 60, sigma_oct, p)
    sw = 1.5 * sigma_oct
    R = int(math.floor(4.5 * sigma_oct + 0.5))
    k = np.arange(-R, R + 1)
    want = m * np.exp(-(k * k) / (2 * sw * sw)).sum() ** 2
    assert abs(hist.sum() - want) / want < 1e-12


@pytest.mark.parametrize("xi", [3, 116])
def test_orientation_window_clipped_at_the_image_edge(xi):
    """Orientation samples need both stencil neighbours, so columns 1..W-2 are
    used: on a ramp the mass is m * (sum of g over the kept columns) * (sum of g
    over all rows), with g(k) = exp(-k^2 / (2 (1.5 sigma)^2)). With sigma = 1.8
    (R = 8) the window at x = 3 loses columns -5..0 and keeps column 1; at
    x = W - 4 it keeps column W - 2."""
    p = so.Params()
    W = 120
    Y, X = np.mgrid[0:121, 0:W].astype(float)
    L = 0.003 * X + 0.004 * Y
    m = 2.0 * math.hypot(0.003, 0.004)
    sig = 1.8
    hist = so.orientation_histogram(L, xi, 60, sig, p)
    sw = 1.5 * sig
    R = int(math.floor(4.5 * sig + 0.5))
    k = np.arange(-R, R + 1)
    g = np.exp(-(k * k) / (2 * sw * sw))
    cols = (xi + k >= 1) & (xi + k <= W - 2)
    assert not cols.all() and (xi + k[cols]).min() in (1, xi - R)
    want = m * g[cols].sum() * g.sum()
    assert abs(hist.sum() - want) / want < 1e-12


@pytest.mark.parametrize("xk", [10.3, 109.6])
def test_descriptor_pixels_clipped_at_the_image_edge(xk):
    """The single-scale descriptor uses pixels 1..W-2 (both stencil neighbours
    inside). On L = x/2 (gradient (1, 0): magnitude 1, all in orientation bin 0)
    at angle 0 the raw mass is separable: (sum over kept columns of g k)(sum over
    rows of g k), offsets from the sub-pixel keypoint in bins of w = 3 sigma,
    g(r) = exp(-r^2 / 8), u = r + 3/2 and k(u) the share of the trilinear split
    inside bins 0..3. With sigma = 2 the support reaches 15 px, past column 1
    (or W - 2)."""
    p = so.Params()
    W, Hh = 120, 121
    Y, X = np.mgrid[0:Hh, 0:W].astype(float)
    L = 0.5 * X
    sig, yk = 2.0, 60.25
    xi, yi = int(round(xk)), 60
    h = so.plain_histogram(L, xk, yk, xi, yi, sig, 0.0, p)
    wbin = 3.0 * sig

    def side(pix, centre, lo, hi):
        r = (pix - centre) / wbin
        u = r + 1.5
        ok = (pix >= lo) & (pix <= hi) & (u > -1) & (u < 4)
        kk = np.where(u < 0, 1 + u, np.where(u > 3, 4 - u, 1.0))
        return (np.exp(-r * r / 8.0) * kk)[ok].sum()

    R = int(math.floor(wbin * math.sqrt(2.0) * 2.5 + 0.5))
    px = np.arange(xi - R, xi + R + 1).astype(float)
    py = np.arange(yi - R, yi + R + 1).astype(float)
    want = side(px, xk, 1, W - 2) * side(py, yk, 1, Hh - 2)
    assert side(px, xk, 1, W - 2) < side(px, xk, -10 ** 6, 10 ** 6)   # the edge cuts the support
    assert h[:, :, 1:].sum() < 1e-12 * h.sum()
    assert h.sum() == pytest.approx(want, rel=1e-12)


def test_orientation_and_descriptor_use_the_nearest_gaussian_level():
    """Orientation and descriptor are taken on the Gaussian level whose scale
    sigma0 2^(i/S) is nearest the keypoint's octave-relative sigma (the
    refined scale offset is below 1/2 level). The level is found here from the
    reported sigma alone, and both results are recomputed on it."""
    img = synth.make_image(synth.rng_for(93, 0), 96, 120)
    p = so.Params()
    res = so.extract(img, p, keep_pyramid=True)
    assert len(res) >= 5
    S = p.n_scales
    for t in range(len(res)):
        o = int(res.octave[t])
        so_t = res.sigma[t] / 2.0 ** o
        i = int(np.argmin([abs(math.log2(so_t / (p.sigma0 * 2.0 ** (k / S)))) for k in range(S + 3)]))
        assert res.layer[t] == i and 1 <= i <= S      # the reported layer is that level
        L = res.pyramid[o][i]
        xi, yi = int(res.internals["xi"][t]), int(res.internals["yi"][t])
        xk, yk = res.x[t] / 2.0 ** o, res.y[t] / 2.0 ** o
        d = so.descriptor(L, xk, yk, xi, yi, so_t, res.angle[t], p)
        np.testing.assert_allclose(res.desc[t], d, atol=1e-12)
        hist = so.orientation_histogram(L, xi, yi, so_t, p)
        angles, _ = so.orientation_peaks(so.smooth_histogram(hist), p)
        assert min(abs((a - res.angle[t] + 180) % 360 - 180) for a in angles) < 1e-9


def test_descriptor_clip_is_active_on_concentrated_mass():
    """Upright on a ramp along a bin centre: all mass sits in one orientation bin and
    the central cells exceed 0.2 of the norm. After clipping, exactly those entries
    are equal to the new maximum, which is below the unclipped maximum."""
    Y, X = np.mgrid[0:121, 0:121].astype(float)
    L = 0.01 * X   # gradient at 0 degrees
    raw = so.descriptor(L, 60.0, 60.0, 60, 60, 2.5, 0.0, so.Params(desc_clip=1.0))
    clp = so.descriptor(L, 60.0, 60.0, 60, 60, 2.5, 0.0, so.Params())
    big = raw > 0.2
    assert big.sum() >= 2 and raw.max() > 0.2
    assert abs(np.linalg.norm(clp) - 1.0) < 1e-12
    np.testing.assert_allclose(clp[big], clp.max(), rtol=1e-12)
    assert np.all(clp[~big] < clp.max())
    assert clp.max() < raw.max()


def test_descriptor_support_is_two_and_a_half_bins_of_three_sigma():
    """READING: spatial bin width w = 3 sigma, samples kept while their rotated
    bin coordinates satisfy |rx|, |ry| < 2.5 (u, v in (-1, 4)). A vertical step
    edge e pixels to the right of the keypoint (angle 0) has gradient only in
    the two pixel columns beside it (central differences, at offsets e - 1 and
    e): with sigma = 2 (w = 6 px) an edge at 12 px lands in spatial column
    floor(rx + 1.5) = 3 with orientation bin 0 only, and one at 17 px lies
    outside the support (rx > 2.5), so the descriptor is zero."""
    p = so.Params()
    n, c, sig = 101, 50, 2.0
    for e, seen in ((12, True), (17, False)):
        L = np.zeros((n, n))
        L[:, c + e:] = 1.0
        d = so.descriptor(L, float(c), float(c), c, c, sig, 0.0, p).reshape(4, 4, 8)
        assert (np.abs(d).sum() > 0) == seen, e
        if seen:
            cols = np.nonzero(d.sum(axis=(0, 2)) > 1e-12)[0].tolist()
            bins = np.nonzero(d.sum(axis=(0, 1)) > 1e-12)[0].tolist()
            assert cols == [3] and bins == [0], (cols, bins)


def test_orientation_peaks_are_strict_maxima():
    """READING: a peak is a strict circular local maximum of the smoothed
    histogram at >= 0.8 of its maximum. A two-bin plateau at the maximum gives
    no peak (neither bin exceeds its neighbour), while a separate strict peak at
    0.9 of the maximum gives one orientation at its bin centre."""
    h = np.zeros(36)
    h[10] = h[11] = 1.0
    h[20] = 0.9
    angles, _ = so.orientation_peaks(h, so.Params())
    assert angles == [200.0]
    h[11] = 0.999                       # break the tie: bin 10 becomes a strict peak
    angles, _ = so.orientation_peaks(h, so.Params())
    assert len(angles) == 2 and abs(angles[1] - 200.0) < 1e-12


def test_orientation_peak_at_exactly_the_ratio_is_kept():
    """READING: a secondary peak is kept at >= 0.8 of the maximum, so one at
    exactly 0.8 (the same double as 0.8 * 1.0) gives a second orientation."""
    h = np.zeros(36)
    h[5] = 1.0
    h[20] = 0.8
    angles, _ = so.orientation_peaks(h, so.Params())
    assert angles == [50.0, 200.0]


def test_descriptor_offsets_from_the_subpixel_keypoint_and_window_reach():
    """READING: sample offsets are taken from the sub-pixel keypoint, and the
    sample window has radius round(w sqrt(2) (d + 1) / 2), which covers the
    rotated 2.5-bin support (w = 3 sigma = 6 px for sigma = 2).
    (a) Angle 0, keypoint 0.4 px right of pixel c, a step whose gradient sits in
        columns c + 15 and c + 16: the first lies 14.6 px = 2.43 bins away,
        inside the support, so the descriptor is not zero.
    (b) Angle 45 degrees, keypoint at pixel c, a step whose gradient sits in
        columns c + 20 and c + 21: the rotated support reaches them (rx, |ry|
        < 2.5 for rows c - 1 .. c + 1), but only a window of radius
        21 = round(6 sqrt(2) 2.5) includes them."""
    p = so.Params()
    n, c, sig = 101, 50, 2.0
    L = np.zeros((n, n))
    L[:, c + 16:] = 1.0
    d = so.descriptor(L, c + 0.4, float(c), c, c, sig, 0.0, p)
    assert np.abs(d).sum() > 0
    L = np.zeros((n, n))
    L[:, c + 21:] = 1.0
    d = so.descriptor(L, float(c), float(c), c, c, sig, 45.0, p)
    assert np.abs(d).sum() > 0


def test_pregate_threshold():
    """READING: candidates need |D| > 0.5 * contrast_thr besides being strict
    3x3x3 extrema: an isolated extremum at 0.4 T is dropped, at 0.6 T kept (both
    signs)."""
    p = so.Params()
    T = p.contrast_thr
    for sign in (1.0, -1.0):
        for frac, n_want in ((0.4, 0), (0.6, 1)):
            D = np.zeros((5, 21, 21))
            D[2, 10, 10] = sign * frac * T
            cs, cy, cx, _, _ = so.find_candidates(D, p)
            assert len(cs) == n_want, (sign, frac)
            if n_want:
                assert (cs[0], cy[0], cx[0]) == (2, 10, 10)


def test_upsampled_outputs_are_in_input_pixels():
    """With the 2x magnified first octave, positions and scales are reported in
    input pixels: a blob centred on input pixel c (magnified pixel 2c, a centre
    of symmetry of the whole pyramid) is found at exactly (c, c), at the scale
    the non-magnified prediction gives in input pixels (the bilinear
    magnification adds a little blur: 3%)."""
    p = so.Params(contrast_thr=0.001, upsample=True)
    s, n = 5.0, 129
    c = n // 2
    Y, X = np.mgrid[0:n, 0:n]
    img = 0.5 + 0.3 * np.exp(-((X - c) ** 2 + (Y - c) ** 2) / (2 * s * s))
    r = so.extract(img, p, with_descriptors=False)
    sel = (np.abs(r.x - c) < 1) & (np.abs(r.y - c) < 1)
    assert sel.any()
    assert np.all(np.abs(r.x[sel] - c) < 1e-9) and np.all(np.abs(r.y[sel] - c) < 1e-9)
    pred = math.sqrt(s * s - p.init_blur ** 2) / math.sqrt(2 ** (1 / 3))
    assert np.all(np.abs(r.sigma[sel] - pred) / pred < 3e-2), (r.sigma[sel], pred)
