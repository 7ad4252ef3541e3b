"""Writes mma_homography_seq0.json: the FP64 oracle's matching accuracy on the
6-image homography sequence (seed index 0, 1000x750, 2x upsampled, cap 8000),
matched by the harness matcher. The GPU accuracy test compares against it.
Calls only the oracle and the workload/harness modules.

    python tests/golden/make_mma_golden.py
"""
import json
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)


def _one(i):
    from oracle import sift_oracle as so
    from workloads import synth
    seq = synth.homography_sequence(0)
    r = so.extract(seq.images[i], so.Params(upsample=True, max_kpts=8000))
    return r.x, r.y, r.desc


class _F:
    def __init__(self, x, y, d):
        import torch
        self.x, self.y, self.desc = torch.tensor(x), torch.tensor(y), torch.tensor(d)


def main():
    from workloads import matching, synth
    seq = synth.homography_sequence(0)
    with mp.get_context("spawn").Pool(min(6, os.cpu_count() or 1)) as pool:
        res = pool.map(_one, range(len(seq.images)))
    acc = matching.sequence_mma([_F(*r) for r in res], seq.homographies)
    acc["keypoints"] = [int(len(r[0])) for r in res]
    acc["what"] = ("FP64 oracle on homography_sequence(0): image 0 matched to images 1-5 "
                   "(mutual NN + ratio 0.8), MMA against the known homographies")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mma_homography_seq0.json")
    with open(out, "w") as f:
        json.dump(acc, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
