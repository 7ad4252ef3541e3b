"""GPU matcher (tcgen05 fp16 similarity, symmetric ratio test) against the
FP64 matcher oracle on the same descriptors. The GPU sums the exact fp16
products in FP32 (error < 1e-5 per similarity), so rows with a decision that a
1e-5 change of a similarity could flip are excluded (the oracle's "robust"
flag); every other row must agree exactly."""
import numpy as np
import pytest

from oracle import matcher as om
from workloads import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2605_17869_gb300 as pkg  # noqa: E402


def _unit(x):
    return (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.float32)


def _planted(seed, na, nb, n_true, noise=0.03):
    rng = np.random.default_rng(seed)
    a = _unit(np.abs(rng.normal(size=(na, 128))) ** 3)
    b = _unit(np.abs(rng.normal(size=(nb, 128))) ** 3)
    perm = rng.permutation(nb)[:n_true]
    b[perm] = _unit(a[:n_true] + noise * np.abs(rng.normal(size=(n_true, 128))))
    return a, b


def _check(a, b, ratio=0.8, max_excluded=0.01):
    ex = pkg.Extractor()
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    got = ex.match(ta, tb, ratio).cpu().numpy()
    got2 = ex.match(ta, tb, ratio).cpu().numpy()
    assert np.array_equal(got, got2)                       # reproducible
    want, info = om.match(a, b, ratio)
    ok = info["robust"]
    bad = np.nonzero(ok & (got != want))[0]
    print(f"na={len(a)} nb={len(b)}: kept gpu {int((got >= 0).sum())} oracle "
          f"{int((want >= 0).sum())}, excluded {int((~ok).sum())}, disagreements {len(bad)}")
    assert len(bad) == 0, bad[:10]
    # Zero descriptors (flat windows) tie exactly with everything; count the
    # excluded rows among the others.
    live = np.linalg.norm(a, axis=1) > 0
    assert (~ok & live).sum() <= max(2, max_excluded * live.sum())
    ex.close()
    return got, want


@pytest.mark.parametrize("na,nb", [(7, 9), (128, 256), (300, 517), (1000, 777), (2100, 2600)])
def test_match_equals_oracle(na, nb):
    n_true = min(na, nb) * 2 // 3
    a, b = _planted(na * 7 + nb, na, nb, n_true)
    got, want = _check(a, b)
    assert (got >= 0).sum() >= 0.9 * n_true


def test_match_degenerate_sizes():
    ex = pkg.Extractor()
    a, b = _planted(3, 5, 6, 4)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    assert np.all(ex.match(ta[:1], tb).cpu().numpy() == -1)   # one descriptor on a side
    assert np.all(ex.match(ta, tb[:1]).cpu().numpy() == -1)
    assert np.all(ex.match(ta, tb[:0]).cpu().numpy() == -1)   # empty set
    assert ex.match(ta[:0], tb).numel() == 0
    with pytest.raises(pkg.SiftError):
        ex.match(ta, tb, ratio=1.5)
    ex.close()


def test_match_real_descriptors_equal_oracle():
    """Descriptors extracted on the GPU from two images of the homography
    sequence, matched on the GPU and by the oracle from the same descriptors."""
    seq = synth.homography_sequence(0)
    ex = pkg.Extractor(upsample=1, max_kpts=8000)
    f = ex.extract_batch([torch.from_numpy(im).cuda() for im in seq.images[:2]])
    a = f[0].desc.cpu().numpy()
    b = f[1].desc.cpu().numpy()
    ex.close()
    got, want = _check(a, b, max_excluded=0.1)
    assert (got >= 0).sum() > 20
