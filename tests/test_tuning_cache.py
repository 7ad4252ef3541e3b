"""Tuning-cache signature and file format (host-only C-ABI calls, no GPU)."""
import json

import pytest

import paper_2605_17869_gb300 as pkg
from paper_2605_17869_gb300 import _abi


def _params(**kw):
    p = _abi.SiftParams()
    pkg._lib().sift_params_default(p)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_signature_ignores_batch_order_but_not_shapes():
    p = _params()
    a = pkg.sift_batch_signature(p, [480, 1200, 600], [640, 1600, 800])
    b = pkg.sift_batch_signature(p, [600, 480, 1200], [800, 640, 1600])
    assert a == b
    assert "n3;" in a and "px2707200;" in a and "side1600;" in a
    # a transposed image, another size or another count: another key
    assert pkg.sift_batch_signature(p, [640, 1200, 600], [480, 1600, 800]) != a
    assert pkg.sift_batch_signature(p, [480, 1200, 601], [640, 1600, 800]) != a
    assert pkg.sift_batch_signature(p, [480, 1200], [640, 1600]) != a


@pytest.mark.parametrize("field,value", [
    ("n_scales", 4), ("sigma0", 1.5), ("upsample", 1), ("contrast_thr", 0.01),
    ("edge_ratio", 12.0), ("border", 6), ("max_kpts", 4096), ("upright", 1), ("dsp", 1),
    ("rootsift", 1), ("upsample_max_px", 1000), ("fp16_pyramid", 1), ("min_octave_side", 32),
])
def test_signature_covers_every_work_parameter(field, value):
    base = pkg.sift_batch_signature(_params(), [480], [640])
    assert pkg.sift_batch_signature(_params(**{field: value}), [480], [640]) != base


def test_signature_rejects_invalid_input():
    with pytest.raises(pkg.SiftError):
        pkg.sift_batch_signature(_params(n_scales=9), [480], [640])
    with pytest.raises(pkg.SiftError):
        pkg.sift_batch_signature(_params(), [0], [640])


def test_cache_round_trip_and_replace(tmp_path):
    path = str(tmp_path / "tuning.json")
    assert pkg.sift_tuning_cache_get(path, "sm103x152;a") is None  # no file yet
    t1 = '{"blur_tile_rows": [[64, 32, 32, 32, 64]], "extrema_ctas_per_sm": 4}'
    t2 = '{"descriptor_ctas_per_sm": 5}'
    pkg.sift_tuning_cache_put(path, "sm103x152;a", t1)
    pkg.sift_tuning_cache_put(path, "sm103x152;b", t2)
    assert pkg.sift_tuning_cache_get(path, "sm103x152;a") == t1
    assert pkg.sift_tuning_cache_get(path, "sm103x152;b") == t2
    assert pkg.sift_tuning_cache_get(path, "sm100x148;a") is None  # other device
    with open(path) as f:
        doc = json.load(f)  # the file is plain JSON
    assert doc["version"] == 1 and set(doc["entries"]) == {"sm103x152;a", "sm103x152;b"}
    assert doc["entries"]["sm103x152;a"]["extrema_ctas_per_sm"] == 4
    pkg.sift_tuning_cache_put(path, "sm103x152;a", t2)  # replaced, not duplicated
    assert pkg.sift_tuning_cache_get(path, "sm103x152;a") == t2
    with open(path) as f:
        assert len(json.load(f)["entries"]) == 2
    assert not [p for p in tmp_path.iterdir() if ".tmp." in p.name]  # no temporary left


def test_cache_refuses_bad_files_and_keys(tmp_path):
    path = tmp_path / "tuning.json"
    path.write_text("{not json")
    with pytest.raises(pkg.SiftError):
        pkg.sift_tuning_cache_get(str(path), "k")
    with pytest.raises(pkg.SiftError):
        pkg.sift_tuning_cache_put(str(path), "k", "{}")
    assert path.read_text() == "{not json"  # left as it was
    path.write_text('{"version": 2, "entries": {}}')
    with pytest.raises(pkg.SiftError):
        pkg.sift_tuning_cache_get(str(path), "k")
    good = str(tmp_path / "good.json")
    for bad_key in ('a"b', "a\\b", "a\nb", ""):
        with pytest.raises(pkg.SiftError):
            pkg.sift_tuning_cache_put(good, bad_key, "{}")
    for bad_json in ("[1, 2]", "{", '{"a": 1} x', "3"):
        with pytest.raises(pkg.SiftError):
            pkg.sift_tuning_cache_put(good, "k", bad_json)
