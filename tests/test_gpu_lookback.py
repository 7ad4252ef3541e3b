"""Bounded waits of the single-pass keypoint compaction, on the GPU.

The candidate and oriented-keypoint compactions are single-pass scans in
which a chunk waits for the counts its predecessors publish. Every wait has a
poll limit; when it runs out the kernel records it and finishes, and the host
reads SIFT_E_TIMEOUT from sift_last_stats. The test makes a wait run out
without any fault: in a child process, the test hook names a chunk that never
publishes and shortens the poll limit. The CUDA context must stay usable and
a handle made without the hook must extract normally in the same process. A
served request whose step gave up carries the same status."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os
import torch
import paper_2605_17869_gb300 as pkg
from workloads import synth

img = torch.from_numpy(synth.make_image(synth.rng_for(51, 0), 600, 800)).cuda()
out = {}
ex = pkg.Extractor(max_kpts=4096)          # reads the hook: chunk 1 never publishes
f = ex.extract(img)
torch.cuda.synchronize()
out["held_count_in_range"] = 0 <= f.count <= 4096
try:
    ex.stats(1)
    out["held_status"] = 0
except pkg.SiftError as e:
    out["held_status"] = e.status
ex.close()
srv = pkg.Server(pkg.Extractor(max_kpts=4096), budget_bytes=1 << 30)  # lanes read the hook too
tk = srv.submit(img)
try:
    srv.result(tk)
    out["served_status"] = 0
except pkg.SiftError as e:
    out["served_status"] = e.status
srv.release(tk)
srv.close()
del os.environ["SIFT_TEST_LOOKBACK_HOLD"]
del os.environ["SIFT_TEST_LOOKBACK_SPINS"]
ex2 = pkg.Extractor(max_kpts=4096)         # no hook
a = ex2.extract(img)
st, rows = pkg.sift_last_stats(ex2.handle, 1)
b = pkg.Extractor(max_kpts=4096).extract(img)
torch.cuda.synchronize()
out["clean_status"] = st
out["clean_count"] = a.count
out["clean_repeatable"] = bool(a.count == b.count and torch.equal(a.desc, b.desc)
                               and torch.equal(a.x, b.x))
print(json.dumps(out))
"""


def test_wait_that_never_completes_reports_timeout_and_context_survives():
    env = dict(os.environ, SIFT_TEST_LOOKBACK_HOLD="1", SIFT_TEST_LOOKBACK_SPINS="2000",
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    import paper_2605_17869_gb300 as pkg
    assert out["held_status"] == pkg.SIFT_E_TIMEOUT
    assert out["served_status"] == pkg.SIFT_E_TIMEOUT  # the serving result carries it too
    assert out["held_count_in_range"]
    assert out["clean_status"] == pkg.SIFT_OK
    assert out["clean_count"] > 0 and out["clean_repeatable"]
