"""GPU MAGSAC++ (through the C ABI) against the FP64 MAGSAC++ oracle on the
same correspondences and the same minimal samples.

The GPU fits each hypothesis in FP64 (elimination instead of the oracle's SVD)
and scores in FP32. The tolerance of a score comes from that arithmetic. Per
correspondence, the FP32 transfer error can be wrong by

    dr <= (dq0 + |px| dq2) / |q2| (same for y),  dq_j = 4 eps T_j,

where T_j is the sum of the absolute terms of row j of H x and eps = 2^-24 (an
unbounded dr when |q2| <= dq2). Its loss can then be wrong by
min(rho_max, s dr), with s the largest slope of the loss within dr of r (zero
past the truncation). A score may differ from the oracle's by twice the sum of
those bounds, plus 1e-5 relative and 1e-3 absolute for the FP32 loss
evaluation and summation. The bound is tight for well-conditioned
models (dr ~ 1e-4 px). It widens only for models that send a correspondence
close to the line at infinity, where FP32 cancels.

Checks:
- the degenerate samples agree exactly;
- every score is within its tolerance;
- the chosen hypothesis ties the oracle's best within their tolerances, and is
  the oracle's best wherever no other hypothesis does;
- its model matches to 1e-7 relative;
- the inlier masks agree except within 1e-3 px (plus dr) of the threshold."""
import numpy as np
import pytest

from oracle import magsac as om
from workloads import synth
from workloads.matching import project

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_17869_gb300 as pkg  # noqa: E402


def _random_h(rng):
    H = np.eye(3)
    H[:2, :2] += rng.normal(scale=0.1, size=(2, 2))
    H[:2, 2] = rng.normal(scale=25.0, size=2)
    H[2, :2] = rng.normal(scale=1e-4, size=2)
    return H


def _planted(seed, n_in, n_out, noise=0.5, size=1000.0):
    rng = np.random.default_rng(seed)
    H = _random_h(rng)
    xa = rng.uniform(0, size, size=(n_in + n_out, 2))
    xb = np.r_[project(H, xa[:n_in]) + rng.normal(scale=noise, size=(n_in, 2)),
               rng.uniform(0, size, size=(n_out, 2))]
    perm = rng.permutation(n_in + n_out)
    return H, xa[perm].astype(np.float32), xb[perm].astype(np.float32)


def _gpu(ex, xa, xb, samples, sigma_max=1.0):
    ta = torch.from_numpy(np.ascontiguousarray(xa)).cuda()
    tb = torch.from_numpy(np.ascontiguousarray(xb)).cuda()
    ts = torch.from_numpy(np.ascontiguousarray(samples.astype(np.int32))).cuda()
    r = ex.magsac(ta, tb, ts, sigma_max=sigma_max)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


EPS32 = 2.0 ** -24


def _dr_bound(Hm, xa, xb):
    """Per-correspondence bound on the FP32 transfer-error error (see above)."""
    p = np.c_[xa.astype(np.float64), np.ones(len(xa))]
    q = p @ Hm.T
    T = np.abs(p) @ np.abs(Hm).T
    dq = 4 * EPS32 * T
    with np.errstate(divide="ignore", invalid="ignore"):
        px, py = q[:, 0] / q[:, 2], q[:, 1] / q[:, 2]
        dx = (dq[:, 0] + np.abs(px) * dq[:, 2]) / np.abs(q[:, 2]) + 4 * EPS32 * (np.abs(px) + 1)
        dy = (dq[:, 1] + np.abs(py) * dq[:, 2]) / np.abs(q[:, 2]) + 4 * EPS32 * (np.abs(py) + 1)
        dr = np.hypot(dx, dy) + 4 * EPS32 * np.abs(xb.astype(np.float64)).sum(axis=1)
    return np.where(np.abs(q[:, 2]) > dq[:, 2], dr, np.inf)


def _score_tol(Hm, xa, xb, score, sigma_max):
    """2 x the sum over correspondences of min(rho_max, s_i dr_i), with s_i the
    largest slope rho'(t) = t w(t) on [r_i - dr_i, r_i + dr_i] (0 past k
    sigma_max; t w(t) rises then falls, so its maximum on an interval is at the
    clamp of its peak t*), plus the evaluation and summation allowance."""
    k = om.chi_quantile() * sigma_max
    t = np.linspace(0.0, k, 4001)
    slope = t * om.weight(t, sigma_max)
    t_peak = t[int(np.argmax(slope))]
    rho_max = float(om.loss(k, sigma_max))
    r = om.residuals(Hm, xa, xb)
    dr = _dr_bound(Hm, xa, xb)
    with np.errstate(invalid="ignore"):
        lo = np.maximum(0.0, np.where(np.isfinite(dr), r - dr, 0.0))
        hi = np.minimum(k, r + dr)
        tc = np.clip(t_peak, lo, np.maximum(lo, hi))
    s_i = np.where(lo < k, tc * om.weight(tc, sigma_max), 0.0)
    with np.errstate(invalid="ignore"):
        per = np.where(np.isfinite(dr), np.minimum(rho_max, s_i * dr), np.where(lo < k, rho_max, 0.0))
    return 2.0 * per.sum() + 1e-5 * abs(score) + 1e-3


def _check(xa, xb, samples, sigma_max=1.0):
    ex = pkg.Extractor()
    g = _gpu(ex, xa, xb, samples, sigma_max)
    g2 = _gpu(ex, xa, xb, samples, sigma_max)
    assert np.array_equal(g["scores"], g2["scores"]) and np.array_equal(g["H"], g2["H"])
    # the oracle sees exactly the FP32 inputs the GPU saw
    H, best, scores, models, inl = om.estimate(xa.astype(np.float64), xb.astype(np.float64),
                                               samples, sigma_max)
    fin = np.isfinite(scores)
    assert np.array_equal(np.isfinite(g["scores"]), fin)
    tol = np.full(len(scores), np.inf)
    for h in np.nonzero(fin)[0]:
        tol[h] = _score_tol(models[h], xa, xb, scores[h], sigma_max)
    err = np.abs(g["scores"][fin].astype(np.float64) - scores[fin])
    assert np.all(err <= tol[fin]), float((err / tol[fin]).max())
    wide = int((tol[fin] > 1e-5 * np.abs(scores[fin]) + 1e-3 + 1e-2).sum())
    print(f"{fin.sum()} valid hypotheses, max err/tol {(err / tol[fin]).max():.3f}, "
          f"{wide} with a widened tolerance")
    gb = int(g["best"][0])
    assert scores[gb] - scores[best] <= tol[gb] + tol[best]
    rivals = fin & (scores - scores[best] <= tol + tol[best])
    if rivals.sum() == 1:
        assert gb == best
    np.testing.assert_allclose(g["H"], models[gb], rtol=1e-7, atol=1e-9)
    r = om.residuals(models[gb], xa, xb)
    k = om.chi_quantile() * sigma_max
    near = np.abs(r - k) < 1e-3 + _dr_bound(models[gb], xa, xb)
    want = r <= k
    assert np.array_equal(g["inliers"].astype(bool)[~near], want[~near])
    ex.close()
    return g, best, scores


@pytest.mark.parametrize("n_in,n_out,n_hyp,sigma_max",
                         [(60, 40, 200, 1.0), (700, 300, 1500, 1.0), (150, 350, 1500, 2.0),
                          (2000, 1000, 1500, 0.75)])
def test_magsac_equals_oracle(n_in, n_out, n_hyp, sigma_max):
    H, xa, xb = _planted(n_in * 13 + n_out, n_in, n_out)
    samples = pkg.draw_samples(len(xa), n_hyp, seed=n_in)
    g, best, _ = _check(xa, xb, samples, sigma_max)
    c = np.array([[0.0, 0.0], [1000.0, 0.0], [1000.0, 1000.0], [0.0, 1000.0]])
    assert np.abs(project(g["H"], c) - project(H, c)).max() < 5.0


def test_magsac_degenerate_and_invalid_inputs():
    ex = pkg.Extractor()
    # all points on one line: every sample is degenerate
    t = np.linspace(0, 100, 50, dtype=np.float32)
    xa = np.c_[t, 2 * t].astype(np.float32)
    g = _gpu(ex, xa, xa + 3, pkg.draw_samples(50, 64, seed=1))
    assert int(g["best"][0]) == -1 and np.isinf(g["score"][0])
    assert not g["inliers"].any() and not g["H"].any()
    # samples with indices outside [0, n) are invalid hypotheses, never read
    H, xa, xb = _planted(3, 30, 10)
    s = pkg.draw_samples(40, 32, seed=2)
    s[::2, 1] = 40 + np.arange(16)
    s[1::4, 3] = -1
    g, _, scores = _check(xa, xb, s)
    assert np.all(np.isinf(g["scores"][::2])) and np.all(np.isinf(g["scores"][1::4]))
    ta = torch.from_numpy(xa).cuda()
    for bad in (dict(sigma_max=0.0), dict(sigma_max=float("nan"))):
        with pytest.raises(pkg.SiftError):
            ex.magsac(ta, ta, n_hyp=8, **bad)
    with pytest.raises(pkg.SiftError):
        ex.magsac(ta[:3], ta[:3], n_hyp=8)
    ex.close()


def test_magsac_on_matched_keypoints():
    """The path end to end on the GPU: extraction, the tensor-core matcher,
    MAGSAC++ on the matched keypoints; the model maps the image corners to
    within 2 px of the known homography, and equals the oracle's choice."""
    seq = synth.homography_sequence(0)
    ex = pkg.Extractor(upsample=1, max_kpts=8000)
    f = ex.extract_batch([torch.from_numpy(im).cuda() for im in seq.images[:2]])
    m = ex.match(f[0].desc, f[1].desc)
    ia = torch.nonzero(m >= 0).flatten()
    ib = m[ia].long()
    xa = torch.stack([f[0].x[ia], f[0].y[ia]], 1).contiguous()
    xb = torch.stack([f[1].x[ib], f[1].y[ib]], 1).contiguous()
    assert xa.shape[0] >= 30
    samples = pkg.draw_samples(xa.shape[0], 1500, seed=0)
    g, best, scores = _check(xa.cpu().numpy(), xb.cpu().numpy(), samples, 1.0)
    h, w = seq.images[0].shape
    c = np.array([[0.0, 0.0], [w, 0.0], [w, h], [0.0, h]])
    err = np.abs(project(g["H"], c) - project(seq.homographies[1], c)).max()
    print(f"{xa.shape[0]} matches, {int(g['inliers'].sum())} inliers, corner error {err:.3f} px")
    assert err < 2.0
    ex.close()
