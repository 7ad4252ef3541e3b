"""FP64 oracle of GPU MAGSAC++ homography verification (test infrastructure only).

Only the test-suite and the benchmark's CPU arms may import this module; the
product path never does, and it shares no code with the CUDA sources.

The paper (§3.6 "GPU MAGSAC++") verifies matches with MAGSAC++ (Barath et al.,
CVPR 2020): 1,500 minimal-sample homography hypotheses, fitted in one batched
SVD and ranked by the soft, noise-marginalised MAGSAC++ score. Everything else
is a READING, written out here from the definitions:

  * samples: hypothesis h uses the 4 correspondences samples[h] (indices drawn
    by the caller; the random draw is an input, so both implementations see
    the same samples); a sample with an index outside [0, n) is invalid;
  * minimal solver: the DLT. Each sample is Hartley-normalised (centroid to the
    origin, mean distance sqrt(2), separately in each image), the 8 x 9 system
    A h = 0 is solved by SVD (right singular vector of the smallest singular
    value), the result is de-normalised and scaled to H[2, 2] = 1;
  * a sample is degenerate (its hypothesis invalid, score +inf) when three of
    its points are collinear in either image (normalised triangle area below
    DEGEN_AREA), when the normalised null vector's last entry is below 1e-9
    (no solution with h33 = 1 in normalised coordinates, the form a minimal
    solver that fixes h33 needs), or when |H[2, 2]| of the de-normalised
    solution is below 1e-12 of its largest entry;
  * residual: forward transfer error r = |pi(H x) - x'| in pixels of the
    second image (pi: division by the third coordinate); a point mapped to
    the line at infinity (third coordinate 0) has r = +inf;
  * score: the MAGSAC++ loss summed over all correspondences, lower is better.
    With the noise sigma of an inlier uniform on [0, sigma_max] and the
    residual of an inlier chi-distributed with n = 4 degrees of freedom
    (noise on the four coordinates of a correspondence), the marginal
    likelihood of a residual t is
        w(t) = C(n) 2^((n-1)/2) / sigma_max * Gamma((n-1)/2, t^2 / (2 sigma_max^2)),
        C(n) = 1 / (2^(n/2) Gamma(n/2)),
    (Gamma(a, x): upper incomplete gamma function). It is truncated at the
    chi quantile k = sqrt(chi2_n^-1(0.99)), shifted to vanish there, and used
    as the IRLS weight of an M-estimator, whose loss is rho(r) = int_0^r t w(t) dt:
        rho(r) = C(n) 2^((n-1)/2) / sigma_max * (sigma_max^2 gamma((n+1)/2, x)
                 + r^2 / 2 * (Gamma((n-1)/2, x) - Gamma((n-1)/2, k^2 / 2))),
        x = r^2 / (2 sigma_max^2), for r <= k sigma_max; rho(k sigma_max) beyond
    (gamma(a, x): lower incomplete gamma). The derivation (substitution
    u = t^2 / (2 sigma^2), then integration by parts) is pinned numerically;
  * the best hypothesis has the smallest score, ties to the smallest index;
    its inliers are the correspondences with r <= k sigma_max. There is no
    local optimisation: the paper names only the hypotheses and the scoring.

Parity status: every function is pinned by tests/test_magsac_oracle.py
(exact recovery from exact correspondences, closed forms against numerical
integration, the chi quantile against a table value, monotonicity and
saturation of the loss, permutation invariance, planted-model recovery).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

DOF = 4                    # READING: degrees of freedom of an inlier's residual
QUANTILE = 0.99            # READING: truncation at the 0.99 chi quantile
DEGEN_AREA = 1e-6          # READING: collinearity threshold (normalised coordinates)
N_HYPOTHESES = 1500        # §3.6: 1,500 minimal-sample hypotheses


def chi_quantile(n: int = DOF, p: float = QUANTILE) -> float:
    """k with P(chi_n <= k) = p: chi^2_n quantile (via the inverse regularised
    lower incomplete gamma function), square-rooted."""
    return math.sqrt(2.0 * special.gammaincinv(n / 2.0, p))


def _upper_gamma(a: float, x):
    """Gamma(a, x), not regularised."""
    return special.gammaincc(a, x) * special.gamma(a)


def _lower_gamma(a: float, x):
    """gamma(a, x), not regularised."""
    return special.gammainc(a, x) * special.gamma(a)


def _c(n: int) -> float:
    return 1.0 / (2.0 ** (n / 2.0) * special.gamma(n / 2.0))


def weight(t, sigma_max: float, n: int = DOF):
    """w(t): the marginal chi_n likelihood of residual t (sigma uniform on
    [0, sigma_max]), shifted to 0 at k sigma_max and 0 beyond."""
    t = np.asarray(t, dtype=np.float64)
    k = chi_quantile(n)
    a = (n - 1) / 2.0
    x = t * t / (2.0 * sigma_max * sigma_max)
    w = _c(n) * 2.0 ** a / sigma_max * (_upper_gamma(a, x) - _upper_gamma(a, k * k / 2.0))
    return np.where(t <= k * sigma_max, w, 0.0)


def loss(r, sigma_max: float, n: int = DOF):
    """rho(r) = int_0^min(r, k sigma_max) t w(t) dt in closed form."""
    r = np.asarray(r, dtype=np.float64)
    k = chi_quantile(n)
    a = (n - 1) / 2.0
    rc = np.minimum(r, k * sigma_max)          # +inf residuals saturate too
    x = rc * rc / (2.0 * sigma_max * sigma_max)
    return _c(n) * 2.0 ** a / sigma_max * (
        sigma_max * sigma_max * _lower_gamma(a + 1.0, x)
        + 0.5 * rc * rc * (_upper_gamma(a, x) - _upper_gamma(a, k * k / 2.0)))


def _normaliser(p: np.ndarray) -> np.ndarray:
    """Hartley: translate the centroid to the origin, scale the mean distance to sqrt(2)."""
    c = p.mean(axis=0)
    d = np.sqrt(((p - c) ** 2).sum(axis=1)).mean()
    s = math.sqrt(2.0) / d if d > 0 else 1.0
    return np.array([[s, 0.0, -s * c[0]], [0.0, s, -s * c[1]], [0.0, 0.0, 1.0]])


def _apply(T: np.ndarray, p: np.ndarray) -> np.ndarray:
    q = np.c_[p, np.ones(len(p))] @ T.T
    return q[:, :2] / q[:, 2:3]


def _collinear(p: np.ndarray) -> bool:
    """Any three of the 4 (normalised) points with triangle area below DEGEN_AREA."""
    for i in range(4):
        for j in range(i + 1, 4):
            for m in range(j + 1, 4):
                a = 0.5 * abs((p[j, 0] - p[i, 0]) * (p[m, 1] - p[i, 1])
                              - (p[j, 1] - p[i, 1]) * (p[m, 0] - p[i, 0]))
                if a < DEGEN_AREA:
                    return True
    return False


def dlt(xa: np.ndarray, xb: np.ndarray):
    """Homography from 4 correspondences xa[j] -> xb[j] (4 x 2 each) by the
    normalised DLT; returns H (3 x 3, H[2, 2] = 1) or None when degenerate."""
    xa = np.asarray(xa, dtype=np.float64)
    xb = np.asarray(xb, dtype=np.float64)
    Ta, Tb = _normaliser(xa), _normaliser(xb)
    pa, pb = _apply(Ta, xa), _apply(Tb, xb)
    if _collinear(pa) or _collinear(pb):
        return None
    A = np.zeros((8, 9))
    for j in range(4):
        x, y = pa[j]
        u, v = pb[j]
        A[2 * j] = [-x, -y, -1.0, 0.0, 0.0, 0.0, u * x, u * y, u]
        A[2 * j + 1] = [0.0, 0.0, 0.0, -x, -y, -1.0, v * x, v * y, v]
    _, _, vt = np.linalg.svd(A)
    v = vt[-1]                                   # unit null vector
    if abs(v[8]) < 1e-9:                         # no solution with h33 = 1 in normalised coordinates
        return None
    Hn = v.reshape(3, 3)
    H = np.linalg.inv(Tb) @ Hn @ Ta
    if abs(H[2, 2]) < 1e-12 * np.abs(H).max():
        return None
    return H / H[2, 2]


def residuals(H: np.ndarray, xa: np.ndarray, xb: np.ndarray) -> np.ndarray:
    """Forward transfer error |pi(H xa) - xb| per correspondence."""
    xa = np.asarray(xa, dtype=np.float64)
    xb = np.asarray(xb, dtype=np.float64)
    q = np.c_[xa, np.ones(len(xa))] @ H.T
    with np.errstate(divide="ignore", invalid="ignore"):
        px = q[:, 0] / q[:, 2]
        py = q[:, 1] / q[:, 2]
        r = np.sqrt((px - xb[:, 0]) ** 2 + (py - xb[:, 1]) ** 2)
    return np.where(q[:, 2] == 0.0, np.inf, r)


def score(H: np.ndarray, xa, xb, sigma_max: float) -> float:
    """MAGSAC++ score of a model: the sum of rho over all correspondences."""
    return float(loss(residuals(H, xa, xb), sigma_max).sum())


def estimate(xa, xb, samples, sigma_max: float = 1.0):
    """Best homography over the hypotheses samples[h] (n_hyp x 4 indices).
    Returns (H, best, scores, models, inliers): scores[h] = +inf for
    degenerate samples; inliers: r <= k sigma_max under the best model."""
    xa = np.asarray(xa, dtype=np.float64)
    xb = np.asarray(xb, dtype=np.float64)
    samples = np.asarray(samples)
    n_hyp = len(samples)
    scores = np.full(n_hyp, np.inf)
    models = np.full((n_hyp, 3, 3), np.nan)
    for h in range(n_hyp):
        idx = samples[h]
        if np.any(idx < 0) or np.any(idx >= len(xa)):   # READING: an invalid sample
            continue
        H = dlt(xa[idx], xb[idx])
        if H is None:
            continue
        models[h] = H
        scores[h] = score(H, xa, xb, sigma_max)
    if not np.isfinite(scores).any():
        return None, -1, scores, models, np.zeros(len(xa), dtype=bool)
    best = int(np.argmin(scores))               # first occurrence: smallest index
    H = models[best]
    inl = residuals(H, xa, xb) <= chi_quantile() * sigma_max
    return H, best, scores, models, inl
