"""Multi-process (gloo, world size 2, CPU) check of the signal sharding used by bench.py."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1509_03979_gb300 import shard


def test_rank_signals_partition():
    W, B = 4, 7
    seen = sorted(i for r in range(W) for i in shard.rank_signals(r, W, B))
    assert seen == list(range(W * B))
    with pytest.raises(ValueError):
        shard.rank_signals(4, 4, 1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        idx = shard.rank_signals(rank, world, 3)
        elapsed = 1.0 + rank            # rank 1 is the slowest
        def reduce_max(x):
            t = torch.tensor([x], dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())
        thr = shard.aggregate_throughput(elapsed, world, 3, 5, reduce_max)
        gathered = [None] * world
        dist.all_gather_object(gathered, idx)
        dist.barrier()
        if rank == 0:
            out.put((gathered, thr))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_disjoint_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, thr = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert gathered == [[0, 1, 2], [3, 4, 5]]
    assert abs(thr - 2 * 3 * 5 / 2.0) < 1e-12       # max elapsed = 2.0 s
