"""The replica path of bench.py (N > 1 ranks, one process each) on CPU with
the gloo backend: every rank's timing is combined by max, and the whole-job
rate counts the units of all ranks over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        rate, slowest = bench.job_rate(100.0, 1.0 + rank, world, dist, torch.device("cpu"))
        total = bench.reduce_scalar(10.0 * (rank + 1), "sum", dist, torch.device("cpu"))
        results[rank] = (rate, slowest, total)
    finally:
        dist.destroy_process_group()


def test_replica_rate_two_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        results = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, results))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(600)  # a spawned rank's first import of torch can take minutes on a cold cache
            assert p.exitcode == 0
        got = dict(results)
    # 2 ranks x 100 units over the slowest rank's 2 s
    for r in range(world):
        rate, slowest, total = got[r]
        assert slowest == 2.0 and rate == 100.0 and total == 30.0


def test_single_rank_needs_no_group():
    import bench
    assert bench.job_rate(50.0, 2.0, 1, None, None) == (25.0, 2.0)
    assert bench.reduce_scalar(3.5, "max", None, None) == 3.5

