"""The parity comparator itself (CPU): an oracle result matched against
perturbed copies of itself finds exactly the keypoints inside each tolerance."""
import math

import numpy as np
import pytest

from oracle import compare
from oracle import sift_oracle as so
from workloads import synth


@pytest.fixture(scope="module")
def ref():
    img = synth.make_image(synth.rng_for(93, 0), 96, 120)
    p = so.Params()
    r = so.extract(img, p, keep_pyramid=True)
    assert len(r) >= 5
    return r, p


def _as_gpu(r):
    return {k: np.array(getattr(r, k), copy=True)
            for k in ("x", "y", "sigma", "angle", "octave", "layer", "desc")}


def test_identical_sets_match_exactly(ref):
    r, p = ref
    m = compare.match(r, _as_gpu(r))
    assert m.n_oracle == len(r) and m.n_eligible == int((r.margin >= compare.MARGIN_EPS).sum())
    assert m.n_found == m.n_eligible > 0 and m.n_excused == m.n_oracle - m.n_eligible
    assert m.n_gpu_unmatched == 0 and m.desc_max_l2 == 0.0
    assert m.worst == {"pos": 0.0, "sigma": 0.0, "angle": 0.0}


@pytest.mark.parametrize("key,delta,found", [
    ("x", 0.005, True), ("x", 0.02, False), ("y", -0.009, True), ("y", -0.011, False),
])
def test_position_tolerance(ref, key, delta, found):
    r, p = ref
    g = _as_gpu(r)
    g[key] = g[key] + delta
    m = compare.match(r, g)
    assert m.n_found == (m.n_eligible if found else 0)
    assert m.n_gpu_unmatched == (0 if found else len(r))
    if found:
        assert m.worst["pos"] == pytest.approx(abs(delta), rel=1e-6)


@pytest.mark.parametrize("rel,found", [(0.5e-3, True), (2e-3, False)])
def test_scale_tolerance(ref, rel, found):
    r, p = ref
    g = _as_gpu(r)
    g["sigma"] = g["sigma"] * (1 + rel)
    m = compare.match(r, g)
    assert m.n_found == (m.n_eligible if found else 0)
    assert m.n_gpu_unmatched == 0          # every GPU keypoint still sits on an oracle keypoint


def test_angle_tolerance_wraps(ref):
    r, p = ref
    g = _as_gpu(r)
    g["angle"] = (g["angle"] + 359.6) % 360.0        # -0.4 degrees, across 0 where it applies
    m = compare.match(r, g)
    assert m.n_found == m.n_eligible
    assert m.worst["angle"] == pytest.approx(0.4, abs=1e-9)
    g["angle"] = (r.angle + 0.6) % 360.0
    assert compare.match(r, g).n_found == 0
    assert compare.angle_diff(359.9, 0.2) == pytest.approx(0.3)


def test_octave_and_layer_must_agree(ref):
    r, p = ref
    g = _as_gpu(r)
    g["layer"] = g["layer"] + 1
    assert compare.match(r, g).n_found == 0
    g = _as_gpu(r)
    g["octave"] = g["octave"] + 1
    assert compare.match(r, g).n_found == 0


def test_keypoints_near_a_threshold_are_excused(ref):
    r, p = ref
    e = np.nonzero(r.margin >= compare.MARGIN_EPS)[0]
    assert len(e) >= 2
    a, b = int(e[0]), int(e[1])                   # two eligible keypoints
    n_el = len(e)
    g = _as_gpu(r)
    keep = np.arange(len(r)) != a
    g = {k: v[keep] for k, v in g.items()}
    m = compare.match(r, g)
    assert m.n_eligible == n_el and m.n_found == n_el - 1
    assert m.n_excused == len(r) - n_el          # a missed keypoint is not an excused one
    saved = r.margin[[a, b]].copy()
    r.margin[a] = 0.5 * compare.MARGIN_EPS
    try:
        m = compare.match(r, g)
        assert m.n_eligible == n_el - 1 and m.n_found == m.n_eligible
        assert m.n_excused == len(r) - n_el + 1
        r.margin[b] = 0.5 * compare.MARGIN_EPS   # excused although present: not counted as found
        m = compare.match(r, g)
        assert m.n_eligible == n_el - 2 and m.n_found == m.n_eligible
    finally:
        r.margin[[a, b]] = saved


def test_descriptor_difference_is_compared_directly(ref):
    """The descriptor difference of a pair is the direct L2 difference of the two
    descriptors. An angle moved within its tolerance still moves the descriptor:
    the comparison reports that difference as it is and never recomputes the
    oracle's descriptor at the GPU's angle."""
    r, p = ref
    g = _as_gpu(r)
    e = np.zeros_like(g["desc"])
    e[:, 0] = 5e-4
    g["desc"] = g["desc"] + e
    m = compare.match(r, g)
    n_el = int((r.margin >= compare.MARGIN_EPS).sum())
    assert m.desc_max_l2 == pytest.approx(5e-4, rel=1e-9) and m.desc_pairs == n_el
    g = _as_gpu(r)
    g["angle"] = (g["angle"] + 0.45) % 360.0
    it = r.internals
    moved = []
    for i in range(len(r)):
        L = r.pyramid[int(r.octave[i])][int(r.layer[i])]
        xi, yi = int(it["xi"][i]), int(it["yi"][i])
        g["desc"][i] = so.descriptor(L, xi + it["dx"][i], yi + it["dy"][i], xi, yi,
                                     it["sigma_oct"][i], float(g["angle"][i]), p)
        if r.margin[i] >= compare.MARGIN_EPS:
            moved.append(float(np.linalg.norm(g["desc"][i] - r.desc[i])))
    m = compare.match(r, g)
    assert m.n_found == n_el
    assert m.desc_max_l2 == pytest.approx(max(moved), rel=1e-12)
    assert m.desc_max_l2 > compare.DESC_TOL


def test_closest_angle_and_worst_case_over_pairs(ref):
    """Among GPU keypoints at the same place within tolerance, the pair uses the
    closest angle; the worst-case figures are maxima over all pairs."""
    r, p = ref
    g = _as_gpu(r)
    twin = {k: v.copy() for k, v in g.items()}
    twin["angle"] = (twin["angle"] + 0.3) % 360.0       # a second orientation, 0.3 degrees off
    both = {k: np.concatenate([g[k], twin[k]]) for k in g}
    m = compare.match(r, both)
    assert m.n_found == m.n_eligible and m.worst["angle"] == 0.0 and m.desc_max_l2 == 0.0
    a = int(np.nonzero(r.margin >= compare.MARGIN_EPS)[0][0])
    g["x"] = g["x"].copy()
    g["x"][a] += 0.005                                    # only one eligible keypoint moves
    m = compare.match(r, g)
    assert m.worst["pos"] == pytest.approx(0.005, rel=1e-6)


def test_tolerance_scale_widens_every_tolerance(ref):
    """tol_scale (the fp16 storage mode's FP16_TOL_SCALE) multiplies the position,
    scale and angle tolerances: offsets 3x outside the FP32 tolerances are
    found at scale 5 and not at scale 1."""
    r, p = ref
    assert compare.FP16_TOL_SCALE == math.ceil(2.0 ** -11 / 1e-4)       # 4.88, rounded up
    for key, delta in (("x", 0.03), ("y", -0.03)):
        g = _as_gpu(r)
        g[key] = g[key] + delta
        assert compare.match(r, g).n_found == 0
        m = compare.match(r, g, tol_scale=compare.FP16_TOL_SCALE)
        assert m.n_found == m.n_eligible > 0
    g = _as_gpu(r)
    g["sigma"] = g["sigma"] * (1 + 3e-3)
    assert compare.match(r, g).n_found == 0
    assert compare.match(r, g, tol_scale=5.0).n_found == compare.match(r, g, tol_scale=5.0).n_eligible
    g = _as_gpu(r)
    g["angle"] = (g["angle"] + 1.5) % 360.0
    assert compare.match(r, g).n_found == 0
    m = compare.match(r, g, tol_scale=5.0)
    assert m.n_found == m.n_eligible
