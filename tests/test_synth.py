"""The seeded input generators follow their stated recipe: deterministic per
seed, in range, with the stated shapes, warps and distributions."""
import math

import numpy as np

from workloads import synth


def test_seeded_and_deterministic():
    a = synth.make_image(synth.rng_for(0, 3), 120, 160)
    b = synth.make_image(synth.rng_for(0, 3), 120, 160)
    c = synth.make_image(synth.rng_for(0, 4), 120, 160)
    assert a.dtype == np.float32 and a.shape == (120, 160)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() <= 1.0
    assert abs(float(a.mean()) - 0.5) < 0.1


def test_fractal_texture_std_and_spectrum():
    """Zero mean, the requested std, and an amplitude spectrum falling as 1/f
    (log-log slope near -1 between 1/64 and 1/4 cycles per pixel)."""
    t = synth.fractal_texture(synth.rng_for(9, 0), 256, 256, std=0.05)
    assert abs(t.std() - 0.05) < 1e-12 and abs(t.mean()) < 1e-12
    amp = np.abs(np.fft.fft2(t))
    fy = np.fft.fftfreq(256)[:, None]
    fx = np.fft.fftfreq(256)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    edges = np.geomspace(1 / 64, 1 / 4, 9)
    mids, means = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        band = (f >= lo) & (f < hi)
        mids.append(math.sqrt(lo * hi))
        means.append(amp[band].mean())
    slope = np.polyfit(np.log(mids), np.log(means), 1)[0]
    assert -1.15 < slope < -0.85, slope


def test_random_homography_ranges_and_centre():
    """Rotation within +-30 degrees and isotropic scale in [0.6, 1.4] about the
    image centre, perspective entries within +-1e-4."""
    rng = synth.rng_for(1, 500)
    h, w = 750, 1000
    c = np.array([(w - 1) / 2.0, (h - 1) / 2.0, 1.0])
    for _ in range(50):
        H = synth.random_homography(rng, h, w)
        q = H @ c
        np.testing.assert_allclose(q[:2] / q[2], c[:2], atol=1e-9)     # the centre is fixed
        T = np.array([[1.0, 0, c[0]], [0, 1.0, c[1]], [0, 0, 1.0]])
        A = np.linalg.inv(T) @ H @ T
        s = math.hypot(A[0, 0], A[1, 0])
        assert 0.6 <= s <= 1.4
        assert abs(math.degrees(math.atan2(A[1, 0], A[0, 0]))) <= 30.0
        assert abs(A[0, 1] + A[1, 0]) < 1e-12 and abs(A[1, 1] - A[0, 0]) < 1e-12   # rotation x scale
        assert np.all(np.abs(A[2, :2]) <= 1e-4)


def test_warp_maps_points_through_the_homography():
    """dst(H p) = src(p) for a smooth image (bilinear interpolation error only)."""
    h, w = 90, 120
    Y, X = np.mgrid[0:h, 0:w].astype(float)
    src = 0.5 + 0.2 * np.sin(X / 9.0) * np.cos(Y / 11.0)
    H = synth.random_homography(synth.rng_for(1, 501), h, w, max_rot_deg=10, scale_range=(0.9, 1.1))
    dst = synth.warp_homography(src, H)
    rng = np.random.default_rng(0)
    for _ in range(50):
        x, y = rng.uniform(30, 90), rng.uniform(25, 65)
        q = H @ np.array([x, y, 1.0])
        u, v = q[0] / q[2], q[1] / q[2]
        iu, iv = int(round(u)), int(round(v))
        q2 = np.linalg.inv(H) @ np.array([iu, iv, 1.0])
        sx, sy = q2[0] / q2[2], q2[1] / q2[2]
        want = 0.5 + 0.2 * math.sin(sx / 9.0) * math.cos(sy / 11.0)
        assert abs(dst[iv, iu] - want) < 2e-3


def test_workload_shapes():
    seq = synth.homography_sequence(0)
    assert len(seq.images) == 6 and all(im.shape == (750, 1000) for im in seq.images)
    np.testing.assert_array_equal(seq.homographies[0], np.eye(3))
    pair = synth.wide_baseline_pair(0)
    assert [im.shape for im in pair.images] == [(1200, 1600)] * 2
    assert synth.single_vga(0).shape == (480, 640)
    shapes = synth.mixed_batch_shapes(200)
    for h, w in shapes:
        long_side, short = max(h, w), min(h, w)
        assert 480 <= long_side <= 1600
        assert any(abs(short - round(long_side * b / a)) == 0 for a, b in ((4, 3), (16, 9)))
    assert any(h > w for h, w in shapes) and any(w > h for h, w in shapes)


def test_serving_trace_distribution():
    """Poisson arrivals (exponential gaps of mean 1/rate) over the three stated
    resolutions in proportions 50 / 35 / 15 %."""
    tr = synth.serving_trace(200.0, 4000)
    t = np.array([r[0] for r in tr])
    gaps = np.diff(np.r_[0.0, t])
    assert np.all(gaps > 0) and abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0
    res = [(r[1], r[2]) for r in tr]
    for hw, p in (((480, 640), 0.50), ((1080, 1920), 0.35), ((2160, 3840), 0.15)):
        assert abs(res.count(hw) / len(res) - p) < 0.03, hw
