"""Matching accuracy of the GPU features on the homography sequence, against
the FP64 oracle's accuracy on the same images (tests/golden/, written by
make_mma_golden.py from the oracle only). Since the GPU keypoints and
descriptors match the oracle's within the parity tolerances, the pooled MMA
and the match count must agree closely."""
import json
import os

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def test_homography_sequence_mma_matches_oracle():
    import paper_2605_17869_gb300 as pkg
    from workloads import matching, synth
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "mma_homography_seq0.json")))
    seq = synth.homography_sequence(0)
    imgs = [torch.from_numpy(im).cuda() for im in seq.images]
    ex = pkg.Extractor(upsample=1, max_kpts=8000)
    feats = ex.extract_batch(imgs)
    acc = matching.sequence_mma(feats, seq.homographies)
    print("gpu", {k: v for k, v in acc.items() if k != "pairs"}, "oracle",
          {k: v for k, v in gold.items() if k.startswith("mma") or k == "matches"})
    # keypoint counts within 2% of the oracle's (near-threshold flips only)
    for n_gpu, n_ref in zip([f.count for f in feats], gold["keypoints"]):
        assert abs(n_gpu - n_ref) <= max(2, 0.02 * n_ref)
    assert abs(acc["matches"] - gold["matches"]) <= max(3, 0.03 * gold["matches"])
    for t in (3, 5, 10):
        assert acc[f"mma@{t}"] >= gold[f"mma@{t}"] - 0.02
    ex.close()
