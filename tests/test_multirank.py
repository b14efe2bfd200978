"""The multi-rank bench logic (one replica per rank, weak scaling, max over
ranks) with world size 2 on the gloo backend, on the CPU."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank 1 is the slow one: the job's time is its time
        t = 0.5 if rank == 1 else 0.25
        m = bench.barrier_max(t, world)
        g = bench.aggregate_gbps(1 << 30, world, t)
        bench.barrier(world)
        q.put((rank, m, g))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, g in got:
        assert m == 0.5
        assert abs(g - 2 * (1 << 30) / 0.5 / 1e9) < 1e-9


def test_single_rank_is_identity():
    import bench
    assert bench.barrier_max(0.125, 1) == 0.125
    assert abs(bench.aggregate_gbps(10 ** 9, 1, 0.5) - 2.0) < 1e-12
