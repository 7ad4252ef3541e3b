"""Multi-GPU host logic of the benchmark (independent replicas), run as two
gloo ranks on CPU: each rank gets its own batch, the timing reduction takes
the maximum over ranks, and the whole-job value divides all ranks' pixels by
that maximum."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    try:
        sys.path.insert(0, ROOT)
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                          WORLD_SIZE=str(world))
        import torch.distributed as dist
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import bench
        m = bench.max_over_ranks(10.0 * (rank + 1), "cpu")
        seq = bench.replica_batch(rank, 2)
        q.put((rank, m, float(seq.images[0].astype("float64").sum()), len(seq.images)))
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, "error", repr(e), 0))


def test_two_gloo_ranks_reduce_max_and_distinct_batches():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    res.sort()
    for r in res:
        assert r[1] != "error", r
    assert [r[1] for r in res] == [20.0, 20.0]        # both ranks see the slowest time
    assert res[0][2] != res[1][2]                      # each rank extracts its own images
    assert [r[3] for r in res] == [2, 2]


def test_whole_job_value_uses_all_ranks_over_slowest():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_value(2, 4.5, 10, 20.0) == pytest.approx(2 * 4.5 * 10 / 0.020)
    assert bench.whole_job_value(1, 4.5, 10, 20.0) == pytest.approx(4.5 * 10 / 0.020)
