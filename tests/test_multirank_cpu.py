"""The N > 1 bench path (replicas only) on CPU: two gloo ranks aggregate their timings the way
bench.py does under torchrun -- the slowest rank's time and the sum of the ranks' updates."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    elapsed = [1.5, 2.25][rank]
    updates = [1e9, 3e9][rank]
    t, u = bench.aggregate_over_ranks(elapsed, updates)
    q.put((rank, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, u in res:
        assert t == pytest.approx(2.25) and u == pytest.approx(4e9)
