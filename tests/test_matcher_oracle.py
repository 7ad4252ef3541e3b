"""Pins for the matcher oracle: brute-force loops, planted pairs, exact
symmetry and permutation invariance, and the degenerate cases."""
import math

import numpy as np
import pytest

from oracle import matcher as om


def _unit(x):
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def _brute(a, b, ratio):
    a = om.round_fp16(a)
    b = om.round_fp16(b)
    out = [-1] * len(a)
    for i in range(len(a)):
        sims = [float(np.dot(a[i], b[j])) for j in range(len(b))]
        order = sorted(range(len(b)), key=lambda j: (-sims[j], j))
        j = order[0]
        d1 = math.sqrt(max(0.0, 2 - 2 * sims[order[0]]))
        d2 = math.sqrt(max(0.0, 2 - 2 * sims[order[1]]))
        back = [float(np.dot(a[k], b[j])) for k in range(len(a))]
        bo = sorted(range(len(a)), key=lambda k: (-back[k], k))
        e1 = math.sqrt(max(0.0, 2 - 2 * back[bo[0]]))
        e2 = math.sqrt(max(0.0, 2 - 2 * back[bo[1]]))
        if bo[0] == i and d1 < ratio * d2 and e1 < ratio * e2:
            out[i] = j
    return np.array(out)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_match_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    a = _unit(np.abs(rng.normal(size=(40, 16))))
    b = _unit(np.abs(rng.normal(size=(50, 16))))
    b[:25] = _unit(a[:25] + 0.05 * np.abs(rng.normal(size=(25, 16))))
    got, _ = om.match(a, b, 0.8)
    np.testing.assert_array_equal(got, _brute(a, b, 0.8))


def test_planted_pairs_recovered_and_symmetric():
    rng = np.random.default_rng(7)
    a = _unit(np.abs(rng.normal(size=(60, 128))))
    perm = rng.permutation(80)
    b = _unit(np.abs(rng.normal(size=(80, 128))))
    b[perm[:60]] = _unit(a + 0.01 * np.abs(rng.normal(size=(60, 128))))
    ab, _ = om.match(a, b)
    ba, _ = om.match(b, a)
    assert np.all(ab == perm[:60])                     # every planted pair found
    for i, j in enumerate(ab):                         # the relation is symmetric
        if j >= 0:
            assert ba[j] == i
    assert (ba >= 0).sum() == (ab >= 0).sum()


def test_permutation_invariance():
    rng = np.random.default_rng(11)
    a = _unit(np.abs(rng.normal(size=(30, 32))))
    b = _unit(np.abs(rng.normal(size=(35, 32))))
    b[:20] = _unit(a[:20] + 0.02)
    pa, pb = rng.permutation(30), rng.permutation(35)
    m0, _ = om.match(a, b)
    m1, _ = om.match(a[pa], b[pb])
    inv_b = np.argsort(pb)
    for k, i in enumerate(pa):
        want = m0[i]
        got = m1[k]
        assert (want < 0 and got < 0) or pb[got] == want


def test_degenerate_cases():
    a = _unit(np.ones((1, 8)))
    b = _unit(np.eye(8))
    m, _ = om.match(a, b)
    assert np.all(m == -1)                             # one descriptor: no ratio test possible
    # Even an exact pair is not kept when one side has a single member: that
    # member has no second neighbour, so its ratio test is undefined.
    m, _ = om.match(b[:1], b)
    assert np.all(m == -1)
    m, _ = om.match(b, b[:1])
    assert np.all(m == -1)
    m, _ = om.match(b, b)
    assert list(m) == list(range(8))                   # each unit vector matches itself (d1 = 0)
    dup = np.vstack([b[:1], b[:1], b[1:3]])
    m, _ = om.match(b[:3], dup)
    assert m[0] == -1                                  # a tie at distance 0 fails 0 < 0.8 * 0
    assert list(m[1:]) == [2, 3]
    x = _unit(np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]]))
    m, _ = om.match(x, x)
    # each vector matches itself; the ratio test: d(x, x) = 0 < 0.8 * second distance
    assert list(m) == [0, 1, 2]


def test_fp16_rounding_reading():
    v = np.array([[0.1, 0.2, 0.3]], dtype=np.float64)
    np.testing.assert_array_equal(om.round_fp16(v), v.astype(np.float16).astype(np.float64))


def test_ties_go_to_the_smaller_index():
    """READING: the nearest neighbour is the largest dot product, ties to the
    smaller index (the match itself never depends on it: a tie fails the ratio
    test, but the reported best indices do)."""
    S = np.array([[1.0, 3.0, 3.0], [2.0, 2.0, 1.0], [0.5, 0.25, 0.5]])
    j1, s1, s2 = om._best_two(S)
    assert list(j1) == [1, 0, 0]
    assert list(s1) == [3.0, 2.0, 0.5] and list(s2) == [3.0, 2.0, 0.5]
    b = _unit(np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]]))
    a = _unit(np.array([[0.1, 1.0, 0.0], [1.0, 0.1, 0.0]]))
    m, info = om.match(a, b)
    assert info["best_a"][0] == 1            # b[1] and b[2] tie: the first wins
    assert m[0] == -1                        # and the tie fails the ratio test


def test_default_ratio_is_lowes():
    """READING: the ratio defaults to Lowe's 0.8. With fp16-exact vectors the
    first row's a-side ratio sqrt(2 - 2 s1) / sqrt(2 - 2 s2), s2 = -1/2, is 0.75
    (s1 = 5/32: kept) or 0.850 (s1 = -43/512: rejected); the other side's test
    and the mutual check pass clearly in both."""
    for s1, kept in ((5 / 32, True), (-43 / 512, False)):
        a = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
        b = np.array([[s1, 0.0, -1.0], [-0.5, 0.0, 0.0]])
        assert np.array_equal(om.round_fp16(b), b)
        m, info = om.match(a, b)
        assert info["best_a"][0] == 0 and info["best_b"][0] == 0
        assert (m[0] == 0) == kept, s1
        assert info["robust"][0]


def test_robust_flags():
    """A row is robust only when every decision behind it keeps its outcome under
    a change of eps in each similarity: a tie between its two best similarities
    is not robust; nor is a ratio test exactly at 0.8 on the other side, with
    d1^2 = 0.64 d2^2 exactly (s1 = 23/64, s2 = -1/1024, all fp16-exact)."""
    a = np.array([[1.0, 0.0, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0]])
    b = np.array([[0.5, 0.5, 0.0, 0.0], [0.5, -0.5, 0.0, 0.0]])
    _, info = om.match(a, b)
    assert info["s1_a"][0] == info["s2_a"][0] and not info["robust"][0]
    a = np.array([[23 / 64, 0.0, 0.0, 0.0], [-1 / 1024, 0.0, 1.0, 0.0]])
    b = np.array([[1.0, 0.0, 0.0, 0.0], [-1.0, 0.0, 0.0, 0.0]])
    _, info = om.match(a, b)
    assert info["best_a"][0] == 0 and info["best_b"][0] == 0
    assert info["s1_b"][0] == 23 / 64 and info["s2_b"][0] == -1 / 1024
    assert not info["robust"][0]
    b[1, 0] = -0.5                                    # a clear case: robust
    a[1, 0] = -0.5
    _, info = om.match(a, b)
    assert info["robust"][0]
