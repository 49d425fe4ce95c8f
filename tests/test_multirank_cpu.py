"""Multi-rank host logic of bench.py (replicas, max-over-ranks time) with two
gloo ranks on CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = 2.0 if rank == 0 else 5.0          # rank 1 is the slow one
    t, v = bench.aggregate_ranks(elapsed, 100.0, dist, "cpu")
    out.put((rank, t, v))
    dist.destroy_process_group()


def test_two_gloo_ranks_use_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 5.0                       # max over ranks
        assert abs(v - 2 * 100.0 / 5.0) < 1e-12   # all ranks' units / slowest time


def test_single_rank_aggregate():
    import bench
    t, v = bench.aggregate_ranks(4.0, 80.0, None)
    assert t == 4.0 and v == 20.0
