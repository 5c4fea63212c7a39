"""The multi-rank path of bench.py on CPU: world_size 2 over gloo.

With --gpus N every rank traverses its own replica of the workload ("replicas only":
the traversal does not shard, so there is no data-path collective).  The whole-job
figure is units_per_rank * N / the slowest rank's time; these tests run the
aggregation functions bench.py uses in two gloo ranks with unequal times.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.job_time(times[rank], world, "cpu")
        q.put((rank, t, bench.whole_job_rate(1_000_000_000, world, t)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(0.5, 2.0), (3.0, 1.0), (1.25, 1.25)])
def test_whole_job_rate_uses_slowest_rank(times):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    slowest = max(times)
    for rank, t, rate in got:
        assert t == pytest.approx(slowest)  # every rank agrees on the job's time
        assert rate == pytest.approx(2 * 1.0 / slowest)  # 2 replicas of 1e9 units each


def test_single_rank_is_local_time():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time(0.75, 1, "cpu") == 0.75
    assert bench.whole_job_rate(3_000_000_000, 1, 1.5) == pytest.approx(2.0)
