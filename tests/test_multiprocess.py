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


def _group_rank(rank, world, port, q):
    """One rank of the shift-group partition on CPU: its partial sum comes
    from the oracle (the library needs a GPU), the partition and the exchange
    step are the product's."""
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import averaging
        from paper_2103_07706_gb300 import shift_groups
        from paper_2103_07706_gb300.inputs import harmonic_state
        from tests.conftest import oracle_model
        m = oracle_model(1, lambda_max=0.00072)
        U, _ = harmonic_state(m.mesh.verts, m.mesh.cells, 2103, 4)
        T, M = 3600.0, 7
        m0, m1 = shift_groups.groups(M, world)[rank]
        part = torch.from_numpy(averaging.averaged_rhs_group(m, T, M, m0, m1, U))
        tot = shift_groups.reduce_partials(part, dist).numpy()
        q.put((rank, tot, m.averaged_rhs(T, M, U) if rank == 0 else None))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_shift_groups_over_two_ranks_reduce_to_the_whole_average():
    """World size 2 over gloo: each rank evaluates its contiguous group of
    shifts, one all-gather exchanges the partial n-vectors, and the sum in
    rank order equals the single-rank average (Sec. 2.5's decomposition)."""
    import numpy as np
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_group_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        r, tot, full = q.get(timeout=300)
        out[r] = (tot, full)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full = out[0][1]
    assert np.array_equal(out[0][0], out[1][0])          # both ranks hold the same sum
    assert np.abs(out[0][0] - full).max() <= 1e-13 * np.abs(full).max()


def test_shift_group_boundaries():
    from paper_2103_07706_gb300 import shift_groups
    assert shift_groups.groups(64, 1) == [(0, 64)]
    g = shift_groups.groups(64, 3)
    assert g[0][0] == 0 and g[-1][1] == 64 and all(a[1] == b[0] for a, b in zip(g, g[1:]))
    assert max(b - a for a, b in g) - min(b - a for a, b in g) <= 1
    with pytest.raises(ValueError):
        shift_groups.groups(2, 3)
