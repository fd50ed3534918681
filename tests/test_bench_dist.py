"""bench.py's multi-rank logic on CPU (gloo, world size 2): the job's rate is
all ranks' units over the slowest rank's time, every rank agrees on it, and
the reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [10.0, 25.0][rank]
    rate, tot = bench.job_rate(1000, ms, world, dist, "cpu")
    # the reference arm returns at once on every rank but 0
    class A:
        steps, warmup, gpus = 1, 0, world
    r = bench.run_reference(A(), None, rank) if rank != 0 else None
    out.put((rank, rate, tot, r))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, rate, tot, r in res:
        assert tot == 25.0
        assert rate == pytest.approx(2 * 1000 / 0.025)
        assert r is None


def test_job_rate_one_rank():
    import bench
    rate, tot = bench.job_rate(500, 20.0, 1)
    assert tot == 20.0 and rate == pytest.approx(500 / 0.02)
