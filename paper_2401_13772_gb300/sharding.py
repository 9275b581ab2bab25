"""Sharding of a batch of independent SP2 parts over ranks (one GPU each).

The parts of a graph-partitioned system are independent problems (§VIII.B),
so the batched path shards by parts and needs no collective on the data path:
each rank solves its own parts in its own persistent launch. Only the timing
(the maximum over ranks) and, optionally, the results cross ranks.

Parts go to ranks by greedy longest-processing-time on the cost n^3 of one
product (every part takes a similar number of iterations): parts in order of
decreasing cost, each to the rank with the least load so far (ties: the lower
rank). The assignment is deterministic, so every rank computes it alone.
"""

from __future__ import annotations


def lpt_shards(costs, world):
    """Indices of the parts of each rank (list of `world` sorted lists)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    loads = [0.0] * world
    shards = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        shards[r].append(i)
        loads[r] += float(costs[i])
    return [sorted(s) for s in shards]


def shard_parts(n, world, rank):
    """Indices (sorted) of the parts of `rank` for parts of orders `n`."""
    if not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    return lpt_shards([float(k) ** 3 for k in n], world)[rank]


def max_over_ranks(value, device=None):
    """The maximum of a float over the ranks of the default process group
    (the value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device=None):
    """The sum of a float over the ranks of the default process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
