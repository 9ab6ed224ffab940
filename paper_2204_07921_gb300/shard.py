"""Sharding independent images across ranks (one process per GPU).

Images are independent units of the sweep, so a batch shards across GPUs
with no collective on the data path: each rank solves its own images and
only the timings (and, if wanted, statistics) are gathered.  A single image
does not shard (coarse blocks straddle any strip split), so it runs as
replicas.

plan_lpt assigns images to ranks by the longest-processing-time rule on a
cost estimate (pixels x an expected cycle count): take images in decreasing
cost, give each to the rank with the least load so far (ties to the lower
rank).  Its makespan is at most 4/3 of the optimum (Graham, 1969).
"""
from __future__ import annotations


def image_cost(H: int, W: int, cycles: float = 1.0) -> float:
    return float(H) * float(W) * float(cycles)


def plan_lpt(costs, n_ranks: int):
    """Returns one list of image indices per rank (each list in increasing
    index order)."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    loads = [0.0] * n_ranks
    parts = [[] for _ in range(n_ranks)]
    for i in order:
        r = min(range(n_ranks), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


def my_share(costs, rank: int, world: int):
    return plan_lpt(costs, world)[rank]
