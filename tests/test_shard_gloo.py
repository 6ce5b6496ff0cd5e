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


def test_balanced_blocks_cover_every_descriptor_once_and_balance_work():
    import numpy as np
    g = np.random.default_rng(1)
    works = list(g.lognormal(0.0, 2.0, size=257))
    for W in (1, 2, 3, 4, 8):
        blocks = shard.balanced_blocks(works, W)
        assert blocks[0][0] == 0 and blocks[-1][1] == len(works)
        assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
        total = sum(works)
        for s, e in blocks:
            assert sum(works[s:e]) <= total / W + max(works) + 1e-9
    assert shard.balanced_blocks([5.0, 5.0, 5.0, 5.0], 2) == [(0, 2), (2, 4)]
    assert sorted(e - s for s, e in shard.balanced_blocks([1.0], 3)) == [0, 0, 1]


def _batch_worker(rank, world, port, out):
    """One rank of the sharded mixed batch, with host-side bookkeeping in place of the GPU
    recovery: the rank's block of the 256 descriptors, a stand-in result per signal, the rank's
    elapsed time proportional to its estimated work, and the max-over-ranks aggregation."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1509_03979_gb300 import synth
        probs = synth.batched_workload(B=256)
        mine = shard.batch_shard(probs, rank, world)
        results = {i: (probs[i].N, probs[i].K) for i in mine}           # stand-in outputs
        work = sum(shard.work_estimate(probs[i].N, probs[i].K, probs[i].algo) for i in mine)
        elapsed = work * 1e-12

        def reduce_max(x):
            t = torch.tensor([x], dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())
        t_max = reduce_max(elapsed)
        gathered = [None] * world
        dist.all_gather_object(gathered, (results, work))
        if rank == 0:
            out.put((gathered, t_max))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_shard_the_mixed_batch_by_work():
    from paper_1509_03979_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, t_max = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    probs = synth.batched_workload(B=256)
    seen = sorted(i for res, _ in gathered for i in res)
    assert seen == list(range(256))                                   # every signal exactly once
    assert all(res[i] == (probs[i].N, probs[i].K) for res, _ in gathered for i in res)
    works = [w for _, w in gathered]
    biggest = max(shard.work_estimate(p.N, p.K, p.algo) for p in probs)
    assert max(works) <= sum(works) / 2 + biggest
    assert abs(t_max - max(works) * 1e-12) < 1e-18
