"""The accuracy harness (mutual-NN + ratio matcher, MMA) checked on CPU against
brute force and planted ground truth."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import matching  # noqa: E402


def _brute(da, db, ratio):
    d = np.sqrt(((da[:, None, :] - db[None, :, :]) ** 2).sum(-1))
    out = set()
    for i in range(da.shape[0]):
        o = np.argsort(d[i], kind="stable")
        j = o[0]
        if not d[i, o[0]] < ratio * d[i, o[1]]:
            continue
        c = np.argsort(d[:, j], kind="stable")
        if c[0] != i or not d[c[0], j] < ratio * d[c[1], j]:
            continue
        out.add((i, int(j)))
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matcher_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    na, nb, n_true = 60, 70, 40
    da = rng.normal(size=(na, 16))
    perm = rng.permutation(nb)[:n_true]
    db = rng.normal(size=(nb, 16))
    db[perm] = da[:n_true] + rng.normal(scale=0.05, size=(n_true, 16))
    ia, ib = matching.mutual_nn_ratio(torch.tensor(da), torch.tensor(db), 0.8)
    got = set(zip(ia.tolist(), ib.tolist()))
    assert got == _brute(da, db, 0.8)
    # every planted pair is recovered (noise is far below the distractor gap)
    assert {(i, int(perm[i])) for i in range(n_true)} <= got


def test_project_and_mma_against_planted_errors():
    th = math.radians(20.0)
    Hm = np.array([[0.9 * math.cos(th), -0.9 * math.sin(th), 30.0],
                   [0.9 * math.sin(th), 0.9 * math.cos(th), -12.0],
                   [1e-5, -2e-5, 1.0]])
    rng = np.random.default_rng(5)
    xy_a = rng.uniform(0, 500, size=(100, 2))
    proj = matching.project(Hm, xy_a)
    # closed form of the projective map for one point
    x, y = xy_a[0]
    den = Hm[2, 0] * x + Hm[2, 1] * y + Hm[2, 2]
    assert proj[0, 0] == pytest.approx((Hm[0, 0] * x + Hm[0, 1] * y + Hm[0, 2]) / den)
    # errors of exactly 2, 4, 8 and 20 px along random directions
    err = np.repeat([2.0, 4.0, 8.0, 20.0], 25)
    ang = rng.uniform(0, 2 * math.pi, 100)
    xy_b = proj + np.stack([err * np.cos(ang), err * np.sin(ang)], 1)
    idx = np.arange(100)
    m, n = matching.mma(xy_a, xy_b, idx, idx, Hm)
    assert n == 100
    assert m["mma@3"] == pytest.approx(0.25)
    assert m["mma@5"] == pytest.approx(0.50)
    assert m["mma@10"] == pytest.approx(0.75)


def test_matcher_handles_tiny_sets():
    ia, ib = matching.mutual_nn_ratio(torch.zeros(1, 4), torch.zeros(5, 4))
    assert ia.numel() == 0 and ib.numel() == 0
