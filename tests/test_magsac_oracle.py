"""Pins for the MAGSAC++ oracle: table values of the chi quantile, the closed
forms of the marginalised weight and loss against numerical integration of
their definitions, exact DLT recovery, degeneracy, permutation invariance and
recovery of a planted homography."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import magsac as om

RNG = np.random.default_rng(20260)


def _project(H, p):
    q = np.c_[p, np.ones(len(p))] @ H.T
    return q[:, :2] / q[:, 2:3]


def _random_h(rng, scale=500.0):
    H = np.eye(3)
    H[:2, :2] += rng.normal(scale=0.1, size=(2, 2))
    H[:2, 2] = rng.normal(scale=0.05 * scale, size=2)
    H[2, :2] = rng.normal(scale=1e-4, size=2)
    return H


def test_chi_quantile_table_values():
    # chi^2 table: 0.99 quantiles 13.277 (4 dof) and 9.210 (2 dof)
    assert abs(om.chi_quantile(4) ** 2 - 13.2767) < 1e-3
    assert abs(om.chi_quantile(2) ** 2 - 9.2103) < 1e-3
    assert abs(om.chi_quantile(4, 0.5) ** 2 - 3.3567) < 1e-3


def _weight_numeric(t, smax, n=om.DOF):
    """Definition: chi_n density of t at noise sigma, averaged over sigma
    uniform on [0, smax]."""
    c = 1.0 / (2.0 ** (n / 2.0) * math.gamma(n / 2.0))
    f = lambda s: 2.0 * c * s ** (-n) * t ** (n - 1) * math.exp(-t * t / (2 * s * s)) / smax
    return integrate.quad(f, 0.0, smax, epsabs=1e-14, epsrel=1e-12, limit=200)[0]


@pytest.mark.parametrize("smax", [0.5, 1.0, 3.0])
def test_weight_closed_form_equals_marginal_integral(smax):
    k = om.chi_quantile()
    shift = _weight_numeric(k * smax, smax)
    for t in np.linspace(0.05, 0.999 * k * smax, 9):
        want = _weight_numeric(t, smax) - shift
        assert abs(float(om.weight(t, smax)) - want) < 1e-10 * max(1.0, abs(want))
    assert float(om.weight(1.01 * k * smax, smax)) == 0.0
    assert abs(float(om.weight(k * smax, smax))) < 1e-15


@pytest.mark.parametrize("smax", [0.5, 1.0, 3.0])
def test_loss_closed_form_equals_integral_of_t_w(smax):
    k = om.chi_quantile()
    for r in np.linspace(0.0, 1.5 * k * smax, 11):
        want = integrate.quad(lambda t: t * float(om.weight(t, smax)), 0.0, min(r, k * smax),
                              epsabs=1e-14, epsrel=1e-12, limit=200)[0]
        assert abs(float(om.loss(r, smax)) - want) < 1e-10 * max(1.0, want)


def test_loss_shape():
    smax = 1.0
    k = om.chi_quantile()
    r = np.linspace(0.0, 3 * k, 400)
    L = om.loss(r, smax)
    assert L[0] == 0.0
    assert np.all(np.diff(L) >= -1e-15)
    top = float(om.loss(k * smax, smax))
    assert np.all(np.abs(L[r >= k] - top) < 1e-15)
    assert float(om.loss(np.inf, smax)) == top
    # near zero rho ~ w(0) r^2 / 2
    w0 = float(om.weight(0.0, smax))
    assert abs(float(om.loss(1e-3, smax)) - 0.5 * w0 * 1e-6) < 1e-9 * w0


def test_dlt_recovers_exact_homography():
    for _ in range(20):
        H = _random_h(RNG)
        xa = RNG.uniform(0, 1000, size=(4, 2))
        xb = _project(H, xa)
        G = om.dlt(xa, xb)
        assert G is not None
        np.testing.assert_allclose(G, H / H[2, 2], rtol=1e-8, atol=1e-10)
        assert np.all(om.residuals(G, xa, xb) < 1e-8)


def test_dlt_degenerate_and_residual_cases():
    xa = np.array([[0.0, 0.0], [100.0, 100.0], [200.0, 200.0], [0.0, 300.0]])  # 3 collinear
    xb = xa + 5.0
    assert om.dlt(xa, xb) is None
    assert om.dlt(xb[[3, 0, 1, 2]], xa[[3, 0, 1, 2]]) is None
    I = np.eye(3)
    p = RNG.uniform(0, 100, size=(5, 2))
    q = RNG.uniform(0, 100, size=(5, 2))
    np.testing.assert_allclose(om.residuals(I, p, q), np.linalg.norm(p - q, axis=1), rtol=1e-15)
    Hinf = np.array([[1.0, 0, 0], [0, 1.0, 0], [1.0, 0, -10.0]])  # x = 10 maps to infinity
    r = om.residuals(Hinf, np.array([[10.0, 3.0], [5.0, 3.0]]), np.zeros((2, 2)))
    assert np.isinf(r[0]) and np.isfinite(r[1])


def test_default_model_has_four_degrees_of_freedom():
    """READING: a correspondence's residual carries the noise of its four
    coordinates, so the defaults are the chi distribution with 4 degrees of
    freedom (0.99 quantile: chi^2 = 13.2767 in the tables) and the weight is
    that of n = 4."""
    assert abs(om.chi_quantile() ** 2 - 13.2767) < 1e-3
    k = om.chi_quantile()
    shift = _weight_numeric(k, 1.0, n=4)
    for t in (0.3, 1.0, 2.5):
        assert abs(float(om.weight(t, 1.0)) - (_weight_numeric(t, 1.0, n=4) - shift)) < 1e-10


def test_hartley_normaliser():
    """Hartley normalisation: the centroid goes to the origin and the mean
    distance from it becomes sqrt(2)."""
    p = RNG.uniform(0, 1000, size=(4, 2))
    q = om._apply(om._normaliser(p), p)
    np.testing.assert_allclose(q.mean(axis=0), 0.0, atol=1e-12)
    assert abs(np.linalg.norm(q, axis=1).mean() - math.sqrt(2.0)) < 1e-12


def test_dlt_degenerate_forms_of_the_minimal_solver():
    """READING of the minimal solver (h33 = 1 in normalised coordinates, then
    H[2, 2] = 1): three collinear points in the second image only, a model that
    sends the first sample's centroid to the line at infinity (normalised
    h33 = 0), and one that sends the image origin there (H[2, 2] = 0) have no
    such solution and are degenerate."""
    xa = np.array([[400.0, 420.0], [610.0, 380.0], [580.0, 600.0], [390.0, 590.0]])
    xb = np.array([[0.0, 0.0], [100.0, 100.0], [200.0, 200.0], [0.0, 300.0]])
    assert om.dlt(xa, xb) is None
    c = xa.mean(axis=0)
    H = np.array([[1.0, 0.1, 5.0], [0.05, 1.0, 3.0], [1e-3, 2e-3, -1e-3 * c[0] - 2e-3 * c[1]]])
    assert om.dlt(xa, _project(H, xa)) is None
    H[2, 2] = 0.0
    assert om.dlt(xa, _project(H, xa)) is None
    H[2, 2] = 1.0                                   # the same model with H[2, 2] = 1 is fine
    G = om.dlt(xa, _project(H, xa))
    assert G is not None
    np.testing.assert_allclose(G, H, rtol=1e-8, atol=1e-10)


def _planted(rng, n_in=150, n_out=100, noise=0.5):
    H = _random_h(rng)
    xa_in = rng.uniform(0, 1000, size=(n_in, 2))
    xb_in = _project(H, xa_in) + rng.normal(scale=noise, size=(n_in, 2))
    xa_out = rng.uniform(0, 1000, size=(n_out, 2))
    xb_out = rng.uniform(0, 1000, size=(n_out, 2))
    xa = np.r_[xa_in, xa_out]
    xb = np.r_[xb_in, xb_out]
    perm = rng.permutation(len(xa))
    truth = np.r_[np.ones(n_in, bool), np.zeros(n_out, bool)][perm]
    return H, xa[perm], xb[perm], truth


def _samples(rng, n, n_hyp):
    return np.array([rng.choice(n, 4, replace=False) for _ in range(n_hyp)])


def _corner_err(H, G, w=1000, h=1000):
    c = np.array([[0.0, 0.0], [w, 0.0], [w, h], [0.0, h]])
    return float(np.abs(_project(H, c) - _project(G, c)).max())


def test_planted_homography_recovered():
    rng = np.random.default_rng(5)
    H, xa, xb, truth = _planted(rng)
    samples = _samples(rng, len(xa), 400)
    G, best, scores, models, inl = om.estimate(xa, xb, samples, sigma_max=1.0)
    assert best == int(np.argmin(scores))
    assert _corner_err(H, G) < 3.0
    assert inl[truth].mean() > 0.95
    assert inl[~truth].mean() < 0.05
    # the true model scores better than the best hypothesis would without it
    assert om.score(H / H[2, 2], xa, xb, 1.0) <= scores[best] * 1.05


def test_scores_invariant_to_correspondence_order_and_ties_to_first():
    rng = np.random.default_rng(9)
    H, xa, xb, _ = _planted(rng, 60, 40)
    samples = _samples(rng, len(xa), 50)
    _, best, s0, _, _ = om.estimate(xa, xb, samples)
    perm = rng.permutation(len(xa))
    inv = np.argsort(perm)
    _, best1, s1, _, _ = om.estimate(xa[perm], xb[perm], inv[samples])
    np.testing.assert_allclose(s1, s0, rtol=1e-12)
    assert best1 == best
    dup = np.r_[samples[best:best + 1], samples]       # the best sample twice
    _, b2, s2, _, _ = om.estimate(xa, xb, dup)
    assert b2 == 0 and s2[0] == s2[best + 1]
    bad = samples.copy()
    bad[0, 2], bad[1, 0] = len(xa), -1                  # indices outside [0, n): invalid
    _, _, s3, _, _ = om.estimate(xa, xb, bad)
    assert np.isinf(s3[0]) and np.isinf(s3[1]) and np.array_equal(s3[2:], s0[2:])
