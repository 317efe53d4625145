"""The multi-rank path of bench.py on CPU: world size 2 over gloo.  Each rank
reports its own time; the job's time is the slowest rank's and its
throughput counts every rank's evaluations (weak scaling, no data-path
collective)."""

import os
import socket

import pytest
import torch.multiprocessing as tmp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms_local = 100.0 * (rank + 1)  # rank 1 is the slow one
        q.put((rank, bench.job_throughput(ms_local, 5, dist, "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_rank_and_count_all_evaluations():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms_max, value = out[r]
        assert ms_max == pytest.approx(200.0)
        assert value == pytest.approx(2 * 5 / 0.2)


def test_single_rank_throughput():
    import bench
    assert bench.job_throughput(250.0, 5) == (250.0, pytest.approx(20.0))
