"""Sharding of independent signals across ranks (one process per GPU).

Signals are independent recoveries, so a batch splits across ranks with no data exchange; the
only collectives are for timing: a barrier around the timed region and a maximum of the
per-rank elapsed times, so the reported throughput is all ranks' signals divided by the
slowest rank's time.  Two partitions:

  * `rank_signals`: rank r of W takes the signals with global index r * B + b, b < B (B signals
    per rank: every rank has the same workload, weak scaling);
  * `balanced_blocks`: a fixed batch of descriptors cut into W contiguous blocks of nearly equal
    estimated work (sum over the block of outer iterations x N log2 N, `work_estimate`), so the
    ranks finish together although per-signal work differs by orders of magnitude.
"""
import math


def rank_signals(rank, world, per_rank):
    """Global indices of the signals rank `rank` recovers."""
    if not (0 <= rank < world) or per_rank < 0:
        raise ValueError("bad rank/world/per_rank")
    return [rank * per_rank + b for b in range(per_rank)]


# Transform applications per outer iteration (estimates of what the device counts): an OMP step is one
# selection plus a warm-started solve (about 6 N-point transforms); an SP round is a merge, two
# solves and two residuals (about 45), over about 6 rounds.
OMP_TRANSFORMS_PER_STEP = 6.0
SP_TRANSFORMS_PER_RUN = 270.0


def work_estimate(N, K, algo):
    """Estimated cost of one recovery: transforms x N log2 N (the cost of one transform)."""
    per = N * math.log2(N)
    if algo == "omp":
        return OMP_TRANSFORMS_PER_STEP * K * per
    return SP_TRANSFORMS_PER_RUN * per


def balanced_blocks(works, world):
    """Cut the descriptor list into `world` contiguous blocks [start, end) whose summed works are
    as even as a contiguous cut allows: block r ends at the prefix sum nearest r/world of the
    total.  Every index lands in exactly one block; a block can be empty only when there are
    fewer descriptors than ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    n = len(works)
    total = float(sum(works))
    cuts = [0]
    run, i = 0.0, 0
    for r in range(1, world):
        target = total * r / world
        while i < n and run + works[i] <= target:
            run += works[i]
            i += 1
        # take one more descriptor when that lands nearer the target
        if i < n and abs(run + works[i] - target) < abs(run - target):
            run += works[i]
            i += 1
        i = max(i, cuts[-1])
        cuts.append(i)
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def aggregate_throughput(elapsed_s, world, per_rank, steps, reduce_max=None):
    """Whole-job signals per second: world * per_rank * steps / max over ranks of elapsed_s.
    `reduce_max(x)` returns the maximum of x over ranks (identity on one rank)."""
    t = reduce_max(elapsed_s) if reduce_max is not None else elapsed_s
    return world * per_rank * steps / t


def batch_shard(descriptors, rank, world):
    """Indices of a fixed batch that rank `rank` of `world` recovers: the balanced contiguous
    block of the descriptor list (each descriptor has N, K and algo)."""
    works = [work_estimate(d.N, d.K, d.algo) for d in descriptors]
    start, end = balanced_blocks(works, world)[rank]
    return list(range(start, end))
