"""Host-side logic of multi-GPU runs: one process per GPU, no data-path collective.

Frames and trajectories are independent (the loss has no cross-frame term), so a multi-GPU
run splits whole trajectories across ranks; the only communication is host-side: a barrier
around the timed region and the maximum of the ranks' times (the job takes as long as its
slowest rank).
"""
from __future__ import annotations

RANK_SEED_STRIDE = 1000  # seed offset between ranks' workloads


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s copy of a workload (rank 0 keeps the base seed)."""
    return int(base) + RANK_SEED_STRIDE * int(rank)


def shard_by_cost(costs, world: int) -> list[list[int]]:
    """Split items (e.g. trajectories, cost = their pair count) over `world` ranks: largest
    first, each to the least-loaded rank. Every item goes to exactly one rank; the result
    lists each rank's item indices in ascending order."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(s) for s in out]


def max_over_ranks(value: float, dist=None) -> float:
    """The largest of the ranks' values (a gloo/NCCL all-reduce of one float64 on the host)."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])
