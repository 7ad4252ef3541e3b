"""The parity comparator itself (CPU): an oracle result matched against
perturbed copies of itself finds exactly the keypoints inside each tolerance."""
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
    m = compare.match(r, _as_gpu(r), params=p)
    assert m.n_found == m.n_eligible == m.n_oracle == len(r)
    assert m.n_gpu_unmatched == 0 and m.desc_max_l2 == 0.0 and m.n_angle_propagated == 0
    assert m.worst == {"pos": 0.0, "sigma": 0.0, "angle": 0.0}


@pytest.mark.parametrize("key,delta,found", [
    ("x", 0.005, True), ("x", 0.02, False), ("y", -0.009, True), ("y", -0.011, False),
])
def test_position_tolerance(ref, key, delta, found):
    r, p = ref
    g = _as_gpu(r)
    g[key] = g[key] + delta
    m = compare.match(r, g, params=p)
    assert m.n_found == (len(r) if found else 0)
    assert m.n_gpu_unmatched == (0 if found else len(r))
    if found:
        assert m.worst["pos"] == pytest.approx(abs(delta), rel=1e-6)


@pytest.mark.parametrize("rel,found", [(0.5e-3, True), (2e-3, False)])
def test_scale_tolerance(ref, rel, found):
    r, p = ref
    g = _as_gpu(r)
    g["sigma"] = g["sigma"] * (1 + rel)
    m = compare.match(r, g, params=p)
    assert m.n_found == (len(r) if found else 0)
    assert m.n_gpu_unmatched == 0          # every GPU keypoint still sits on an oracle keypoint


def test_angle_tolerance_wraps(ref):
    r, p = ref
    g = _as_gpu(r)
    g["angle"] = (g["angle"] + 359.6) % 360.0        # -0.4 degrees, across 0 where it applies
    m = compare.match(r, g, params=p)
    assert m.n_found == len(r)
    assert m.worst["angle"] == pytest.approx(0.4, abs=1e-9)
    g["angle"] = (r.angle + 0.6) % 360.0
    assert compare.match(r, g, params=p).n_found == 0
    assert compare.angle_diff(359.9, 0.2) == pytest.approx(0.3)


def test_octave_and_layer_must_agree(ref):
    r, p = ref
    g = _as_gpu(r)
    g["layer"] = g["layer"] + 1
    assert compare.match(r, g, params=p).n_found == 0
    g = _as_gpu(r)
    g["octave"] = g["octave"] + 1
    assert compare.match(r, g, params=p).n_found == 0


def test_keypoints_near_a_threshold_are_excused(ref):
    r, p = ref
    g = _as_gpu(r)
    keep = np.arange(len(r)) != 0
    g = {k: v[keep] for k, v in g.items()}
    m = compare.match(r, g, params=p)
    assert m.n_found == m.n_eligible - 1
    saved = r.margin[:2].copy()
    r.margin[0] = 0.5 * compare.MARGIN_EPS
    try:
        m = compare.match(r, g, params=p)
        assert m.n_eligible == len(r) - 1 and m.n_found == m.n_eligible
        r.margin[1] = 0.5 * compare.MARGIN_EPS   # excused although present: not counted as found
        m = compare.match(r, g, params=p)
        assert m.n_eligible == len(r) - 2 and m.n_found == m.n_eligible
    finally:
        r.margin[:2] = saved


def test_descriptor_difference_and_angle_propagation(ref):
    r, p = ref
    g = _as_gpu(r)
    e = np.zeros_like(g["desc"])
    e[:, 0] = 5e-4
    g["desc"] = g["desc"] + e
    m = compare.match(r, g, params=p)
    assert m.desc_max_l2 == pytest.approx(5e-4, rel=1e-9) and m.desc_pairs == len(r)
    # The angle moved inside its tolerance, the descriptor computed at the moved
    # angle: the direct difference is large, the one at the GPU angle is zero.
    g = _as_gpu(r)
    g["angle"] = (g["angle"] + 0.45) % 360.0
    it = r.internals
    for i in range(len(r)):
        L = r.pyramid[int(r.octave[i])][int(r.layer[i])]
        xi, yi = int(it["xi"][i]), int(it["yi"][i])
        g["desc"][i] = so.descriptor(L, xi + it["dx"][i], yi + it["dy"][i], xi, yi,
                                     it["sigma_oct"][i], float(g["angle"][i]), p)
    m = compare.match(r, g, params=p)
    assert m.desc_max_l2_direct > compare.DESC_TOL
    assert m.desc_max_l2 < 1e-12
    assert m.n_angle_propagated >= 1


def test_closest_angle_and_worst_case_over_pairs(ref):
    """Among GPU keypoints at the same place within tolerance, the pair uses the
    closest angle; the worst-case figures are maxima over all pairs."""
    r, p = ref
    g = _as_gpu(r)
    twin = {k: v.copy() for k, v in g.items()}
    twin["angle"] = (twin["angle"] + 0.3) % 360.0       # a second orientation, 0.3 degrees off
    both = {k: np.concatenate([g[k], twin[k]]) for k in g}
    m = compare.match(r, both, params=p)
    assert m.n_found == len(r) and m.worst["angle"] == 0.0 and m.desc_max_l2 == 0.0
    g["x"] = g["x"].copy()
    g["x"][0] += 0.005                                    # only the first keypoint moves
    m = compare.match(r, g, params=p)
    assert m.worst["pos"] == pytest.approx(0.005, rel=1e-6)
