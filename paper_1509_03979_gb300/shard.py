"""Sharding of independent signals across ranks (one process per GPU).

Signals are independent recoveries, so a batch splits across ranks with no data exchange: rank r
of W takes the signals with global index i = r * B + b, b < B (B signals per rank, weak
scaling).  The only collectives are for timing: a barrier around the timed region and a
maximum of the per-rank elapsed times, so the reported throughput is all ranks' signals divided
by the slowest rank's time.
"""


def rank_signals(rank, world, per_rank):
    """Global indices of the signals rank `rank` recovers."""
    if not (0 <= rank < world) or per_rank < 0:
        raise ValueError("bad rank/world/per_rank")
    return [rank * per_rank + b for b in range(per_rank)]


def aggregate_throughput(elapsed_s, world, per_rank, steps, reduce_max=None):
    """Whole-job signals per second: world * per_rank * steps / max over ranks of elapsed_s.
    `reduce_max(x)` returns the maximum of x over ranks (identity on one rank)."""
    t = reduce_max(elapsed_s) if reduce_max is not None else elapsed_s
    return world * per_rank * steps / t
