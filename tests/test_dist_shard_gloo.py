"""Row-sharded march on two gloo ranks (CPU): each rank holds half of the rows of every T_k and of
T_0^-1, forms its rows of b_n without communication, and all-gathers b_n and y_n each step
(paper_2312_06367_gb300/shard.py).  The two-rank march must equal the one-rank march bit for bit
(FP64), and the dense MOT recurrence of the oracle (LU solve) to rounding."""
import os
import socket
import sys
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _march(path, rank, world, allgather):
    sys.path.insert(0, ROOT)
    from paper_2312_06367_gb300.shard import ShardedMarch, row_ranges
    d = np.load(path)
    T, T0inv, r = d["T"], d["T0inv"], d["r"]
    n, R = r.shape[1], r.shape[2]
    lo, hi = row_ranges(n, world, tile=32)[rank]
    m = ShardedMarch(T[:, lo:hi], T0inv[lo:hi], lo, hi, n, R, allgather)
    return np.stack([m.step(r[i, lo:hi]) for i in range(r.shape[0])])


def _rank(rank, world, port, path, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2312_06367_gb300.shard import row_ranges
    n = np.load(path)["r"].shape[1]
    ranges = row_ranges(n, world, tile=32)
    width = max(b - a for a, b in ranges)

    def allgather(local):
        buf = torch.zeros((width, local.shape[1]), dtype=torch.float64)
        buf[:local.shape[0]] = torch.from_numpy(local)
        parts = [torch.zeros_like(buf) for _ in range(world)]
        dist.all_gather(parts, buf)
        return np.concatenate([p[:b - a].numpy() for p, (a, b) in zip(parts, ranges)])

    y = _march(path, rank, world, allgather)
    if rank == 0:
        q.put(y)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_row_ranges_cover_on_tiles():
    sys.path.insert(0, ROOT)
    from paper_2312_06367_gb300.shard import row_ranges
    for n, world in ((7680, 8), (120, 2), (1000, 3), (5, 4)):
        rr = row_ranges(n, world)
        assert rr[0][0] == 0 and rr[-1][1] == n
        assert all(a == b0 for (_, a), (b0, _) in zip(rr[:-1], rr[1:]))
        assert all(a % 128 == 0 for a, _ in rr)


def test_two_rank_row_sharded_march_is_bit_exact(ico1_ops, ico1_fm):
    import torch.multiprocessing as mp
    from oracle import mot, rhs
    from synth import excitation
    nt = 40
    pw = excitation.random_batch(2, seed=21, t0=4.0, sigma=1.5)
    e, h = rhs.incident_tests(ico1_ops, pw, ico1_ops.dt * np.arange(1, nt + 1))
    r = ico1_fm.rhs(e, h)
    T = ico1_fm.T_stack()
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "march.npz")
        np.savez(path, T=T, T0inv=np.linalg.inv(T[0]), r=r)
        one = _march(path, 0, 1, lambda x: x)
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(k, 2, port, path, q)) for k in range(2)]
        for p in procs:
            p.start()
        two = q.get(timeout=300)
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
    assert np.array_equal(one, two)
    ref = mot.march_dense(T, r)
    assert np.linalg.norm(two - ref) <= 1e-12 * np.linalg.norm(ref)
