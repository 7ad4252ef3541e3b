"""The identity the magnified base kernel is built on (CPU, FP64): the base
blur of the 2x bilinear magnification, blur(upsample2x(I)) with reflect-101 on
the magnified grid, equals a two-phase filter of the input itself. Output
sample 2k + p is sum_q c_p[q] I_e[k + q], where c_p[q] collects the base taps
that land on input sample k + q through the magnification, and I_e is the
input extended by I_e[i] = I[refl101(2i, 2n) / 2]. This holds exactly,
borders included, for any size. Both sides are computed here from the oracle's
own functions and taps; nothing is shared with the CUDA code."""
import numpy as np
import pytest

from oracle import sift_oracle as so


def _refl101(i, n):
    i = -i if i < 0 else i
    return 2 * n - 2 - i if i >= n else i


def _phase_taps(w, R):
    Q = (R + 2) // 2
    c = np.zeros((2, 2 * Q + 1))
    for p in range(2):
        for t in range(-R, R + 1):
            m = p + t                      # magnified offset from 2k
            if m % 2 == 0:
                c[p, m // 2 + Q] += w[t + R]
            else:
                c[p, (m - 1) // 2 + Q] += 0.5 * w[t + R]
                c[p, (m + 1) // 2 + Q] += 0.5 * w[t + R]
    return c, Q


def _polyphase(img, w, R):
    h, wd = img.shape
    c, Q = _phase_taps(w, R)
    rows = [_refl101(2 * i, 2 * h) // 2 for i in range(-Q, h + Q)]
    cols = [_refl101(2 * i, 2 * wd) // 2 for i in range(-Q, wd + Q)]
    ext = img[np.ix_(rows, cols)]                      # I_e on [-Q, n + Q)
    tmp = np.zeros((ext.shape[0], 2 * wd))             # rows filtered to the magnified width
    for k in range(wd):
        for p in range(2):
            tmp[:, 2 * k + p] = ext[:, k:k + 2 * Q + 1] @ c[p]
    out = np.zeros((2 * h, 2 * wd))
    for k in range(h):
        for p in range(2):
            out[2 * k + p] = c[p] @ tmp[k:k + 2 * Q + 1]
    return out


@pytest.mark.parametrize("shape", [(8, 8), (9, 13), (16, 11), (31, 40)])
@pytest.mark.parametrize("sigma0", [1.6, 2.0])
def test_polyphase_equals_blur_of_magnification(shape, sigma0):
    rng = np.random.default_rng(shape[0] * 100 + shape[1])
    img = rng.random(shape)
    p = so.Params(upsample=True, sigma0=sigma0)
    sb = so.base_sigma(p)
    R, w = so.gaussian_taps(sb)
    want = so.blur(so.upsample2x(img), sb)
    got = _polyphase(img, w, R)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def test_phase_taps_sum_to_one():
    R, w = so.gaussian_taps(so.base_sigma(so.Params(upsample=True)))
    c, Q = _phase_taps(w, R)
    assert Q == (R + 2) // 2
    np.testing.assert_allclose(c.sum(axis=1), [1.0, 1.0], atol=1e-15)
