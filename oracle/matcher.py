"""FP64 oracle of the symmetric ratio-test matcher (test infrastructure only).

Only the test-suite and the benchmark's CPU arms may import this module; the
product path never does, and it shares no code with the CUDA sources.

The paper's first matching backend (§3.4 "Descriptor Matching") forms the
similarity matrix of two descriptor sets with fp16 tensor-core products and
keeps mutually consistent pairs that pass a ratio test. Readings where the
paper is silent (marked READING):
  * the operands are the descriptors rounded to fp16 (the precision the paper
    names); products and sums here are exact in FP64 (the GPU sums fp16
    products in FP32, which only matters within ~1e-5 of a tie);
  * the nearest neighbour is the largest dot product, ties to the smaller
    index; descriptors are unit vectors, so the Euclidean distance is
    d = sqrt(max(0, 2 - 2 s));
  * a pair (i, j) is kept when j is i's nearest neighbour, i is j's, and both
    pass Lowe's ratio test d1 < ratio * d2 (ratio 0.8 by default) among their
    own candidates; a set with a single member has no second neighbour and
    keeps nothing.

Parity status: match is pinned by tests/test_matcher_oracle.py (brute-force
loops, planted pairs, symmetry and permutation invariance, the default ratio
and the robustness flags on fp16-exact vectors, single-member sets).
"""
from __future__ import annotations

import numpy as np


def round_fp16(x: np.ndarray) -> np.ndarray:
    """READING: the matcher's operands are the descriptors rounded to fp16."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float64)


def _best_two(S: np.ndarray):
    """Per row of S: index of the largest entry (ties: smallest index), the
    largest and the second largest value (over the other columns)."""
    n, m = S.shape
    j1 = np.argmax(S, axis=1)                      # first occurrence = smallest index
    s1 = S[np.arange(n), j1]
    T = S.copy()
    T[np.arange(n), j1] = -np.inf
    s2 = T.max(axis=1) if m > 1 else np.full(n, -np.inf)
    return j1, s1, s2


def distance(s: np.ndarray) -> np.ndarray:
    """Euclidean distance of unit vectors with dot product s."""
    return np.sqrt(np.maximum(0.0, 2.0 - 2.0 * s))


def _ratio_robust(s1: float, s2: float, ratio: float, eps: float) -> bool:
    """d(s1) < ratio * d(s2) has the same truth value for every s1', s2' within
    eps of s1, s2 (d decreases in s, so the extremes decide)."""
    lo = distance(np.array([s1 + eps]))[0] < ratio * distance(np.array([s2 - eps]))[0]
    hi = distance(np.array([s1 - eps]))[0] < ratio * distance(np.array([s2 + eps]))[0]
    return bool(lo == hi)


def match(desc_a: np.ndarray, desc_b: np.ndarray, ratio: float = 0.8, eps: float = 1e-5):
    """Returns (match_a, info): match_a[i] = j for every kept pair (i, j), else
    -1; info holds the per-row decision quantities (best index, the two best
    similarities of each side) and info["robust"][i]: whether every decision
    that concerns row i (its nearest neighbour j, j's nearest neighbour, and
    both ratio tests) keeps its outcome when each similarity involved moves by
    up to eps. A GPU that sums the (exact) fp16 products in FP32 errs by less
    than 128 * 2^-24 ~ 7.6e-6 per similarity, so with eps = 1e-5 its result
    must equal the oracle's on every robust row."""
    a = round_fp16(desc_a)
    b = round_fp16(desc_b)
    na, nb = a.shape[0], b.shape[0]
    out = np.full(na, -1, dtype=np.int64)
    info = {"robust": np.ones(na, dtype=bool)}
    if na < 2 or nb < 2:
        return out, info
    S = a @ b.T
    ja, sa1, sa2 = _best_two(S)        # for each i in a: best j
    ib, sb1, sb2 = _best_two(S.T)      # for each j in b: best i
    da1, da2 = distance(sa1), distance(sa2)
    db1, db2 = distance(sb1), distance(sb2)
    for i in range(na):
        j = ja[i]
        keep = ib[j] == i and da1[i] < ratio * da2[i] and db1[j] < ratio * db2[j]
        if keep:
            out[i] = j
        info["robust"][i] = (_ratio_robust(sa1[i], sa2[i], ratio, eps)
                             and _ratio_robust(sb1[j], sb2[j], ratio, eps)
                             and sa1[i] - sa2[i] > 2 * eps and sb1[j] - sb2[j] > 2 * eps)
    info.update(best_a=ja, s1_a=sa1, s2_a=sa2, best_b=ib, s1_b=sb1, s2_b=sb2)
    return out, info
