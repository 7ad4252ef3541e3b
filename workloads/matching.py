"""Accuracy harness for the homography workloads: descriptor matching and
mean matching accuracy (MMA) against the known homography.

This is measurement, not part of the extractor: a brute-force mutual nearest
neighbour matcher with Lowe's ratio test, written with plain torch tensor
operations, and the fraction of matches whose keypoint lands within t pixels
of where the homography maps its partner (MMA@t), the usual accuracy figure
for homography sequences.
"""
from __future__ import annotations

import numpy as np


def mutual_nn_ratio(desc_a, desc_b, ratio: float = 0.8):
    """Indices (ia, ib) of pairs that are mutual nearest neighbours in L2 and
    pass the ratio test d1 < ratio * d2 in both directions. desc_* are
    (N, D) float tensors on any device; returns int64 tensors on that device."""
    import torch  # noqa: PLC0415

    na, nb = desc_a.shape[0], desc_b.shape[0]
    if na < 2 or nb < 2:
        e = torch.zeros(0, dtype=torch.int64, device=desc_a.device)
        return e, e
    d = torch.cdist(desc_a.double(), desc_b.double())
    va, ia = torch.topk(d, 2, dim=1, largest=False)   # best two in b for each a
    vb, ib = torch.topk(d, 2, dim=0, largest=False)   # best two in a for each b
    nn_ab = ia[:, 0]
    nn_ba = ib[0, :]
    a_idx = torch.arange(na, device=d.device)
    mutual = nn_ba[nn_ab] == a_idx
    ok_a = va[:, 0] < ratio * va[:, 1]
    ok_b = vb[0, :] < ratio * vb[1, :]
    keep = mutual & ok_a & ok_b[nn_ab]
    return a_idx[keep], nn_ab[keep]


def project(Hm: np.ndarray, xy: np.ndarray) -> np.ndarray:
    """Apply a 3x3 homography to (N, 2) points (x, y)."""
    p = np.concatenate([xy, np.ones((xy.shape[0], 1))], axis=1) @ np.asarray(Hm, np.float64).T
    return p[:, :2] / p[:, 2:3]


def mma(xy_a: np.ndarray, xy_b: np.ndarray, ia: np.ndarray, ib: np.ndarray, Hm: np.ndarray,
        thresholds=(3, 5, 10)):
    """MMA@t: fraction of matches (ia[k], ib[k]) with |H xy_a - xy_b| <= t px,
    where Hm maps image-a pixel coordinates to image-b coordinates."""
    if len(ia) == 0:
        return {f"mma@{t}": 0.0 for t in thresholds}, 0
    err = np.linalg.norm(project(Hm, xy_a[ia]) - xy_b[ib], axis=1)
    return {f"mma@{t}": float(np.mean(err <= t)) for t in thresholds}, int(len(ia))


def sequence_mma(feats, homographies, thresholds=(3, 5, 10), ratio: float = 0.8):
    """Pooled MMA of image 0 matched against each image k >= 1 of a sequence.
    feats[k] has .x, .y (tensors) and .desc (N x 128 tensor)."""
    hits = {t: 0 for t in thresholds}
    total = 0
    per_pair = []
    xy0 = np.stack([feats[0].x.cpu().numpy(), feats[0].y.cpu().numpy()], 1).astype(np.float64)
    for k in range(1, len(feats)):
        ia, ib = mutual_nn_ratio(feats[0].desc, feats[k].desc, ratio)
        ia, ib = ia.cpu().numpy(), ib.cpu().numpy()
        xyk = np.stack([feats[k].x.cpu().numpy(), feats[k].y.cpu().numpy()], 1).astype(np.float64)
        m, n = mma(xy0, xyk, ia, ib, homographies[k], thresholds)
        per_pair.append({"image": k, "matches": n, **{kk: round(v, 4) for kk, v in m.items()}})
        for t in thresholds:
            hits[t] += round(m[f"mma@{t}"] * n)
        total += n
    pooled = {f"mma@{t}": round(hits[t] / total, 4) if total else 0.0 for t in thresholds}
    return {"matches": total, **pooled, "pairs": per_pair}
