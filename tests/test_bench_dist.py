"""The N > 1 replica path of bench.py on CPU ranks (gloo, world size 2): the
timed region's result is the slowest rank's time, and the value is the
whole-job throughput (units of every rank over that time)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    elapsed = 1.0 + rank  # rank 1 is slower
    t, v = bench.aggregate(elapsed, 1000.0, dist)
    q.put((rank, t, v))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_max_time_and_sum_units():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 2.0
        assert v == 1000.0 * 2 / 2.0


def test_single_process_aggregate():
    import bench
    t, v = bench.aggregate(0.5, 100.0, None)
    assert t == 0.5 and v == 200.0
