"""The N > 1 bench path on CPU: two gloo ranks stand in for two GPUs (replicas, no data-path
collective).  The whole-job rate counts every rank's steps over the slowest rank's time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, ws, port, times, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    value, tot = bench.whole_job_rate(times[rank], 50, ws, dist, "cpu")
    q.put((rank, value, tot))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("times", [(100.0, 250.0), (80.0, 80.0)])
def test_whole_job_rate_two_gloo_ranks(times):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slow = max(times)
    for _, value, tot in got:
        assert tot == slow                        # every rank sees the slowest rank's time
        assert abs(value - 2 * 50 / (slow / 1e3)) < 1e-9 * value


def test_whole_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    value, tot = bench.whole_job_rate(200.0, 100, 1)
    assert tot == 200.0 and abs(value - 500.0) < 1e-12
