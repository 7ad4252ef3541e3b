"""Host logic of the MAGSAC++ binding: draw_samples gives every hypothesis 4
distinct indices in [0, n), uniformly, reproducibly for a seed (CPU only)."""
import itertools

import numpy as np
import pytest

import paper_2605_17869_gb300 as pkg


def test_rows_are_distinct_in_range_and_seeded():
    s = pkg.draw_samples(37, 5000, seed=3)
    assert s.dtype == np.int32 and s.shape == (5000, 4)
    assert s.min() >= 0 and s.max() < 37
    assert all(len(set(r)) == 4 for r in s.tolist())
    assert np.array_equal(s, pkg.draw_samples(37, 5000, seed=3))
    assert not np.array_equal(s, pkg.draw_samples(37, 5000, seed=4))


def test_uniform_over_subsets_and_positions():
    n, m = 6, 60000
    s = pkg.draw_samples(n, m, seed=11)
    # every index equally likely in every position: chi-square over 6 cells
    for k in range(4):
        c = np.bincount(s[:, k], minlength=n)
        chi2 = ((c - m / n) ** 2 / (m / n)).sum()
        assert chi2 < 25.0, (k, c)          # 5 dof: P(chi2 > 25) < 2e-4
    # every ordered 4-tuple of distinct indices equally likely (360 cells)
    keys = {t: i for i, t in enumerate(itertools.permutations(range(n), 4))}
    c = np.bincount([keys[tuple(r)] for r in s.tolist()], minlength=len(keys))
    e = m / len(keys)
    chi2 = ((c - e) ** 2 / e).sum()
    assert chi2 < 359 + 6 * np.sqrt(2 * 359), chi2   # mean 359, 6 standard deviations


def test_small_sets():
    s = pkg.draw_samples(4, 200, seed=0)
    assert all(sorted(r) == [0, 1, 2, 3] for r in s.tolist())
    with pytest.raises(pkg.SiftError):
        pkg.draw_samples(3, 10)
