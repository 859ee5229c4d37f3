"""Source sharding across ranks (one process per GPU).

Sec. 4.4: J p concatenates the per-source products and J^T y sums them,
J^T y = sum_a J_a^T y_a.  With sources split across ranks, J needs no exchange and J^T
needs one sum of the model-space result over ranks (the distributed accumulation of
Sec. 5.3).  Sources are assigned greedily by cost (longest first to the least loaded
rank); the cost of a source is its node-updates times its level count, the two factors
that set its traversal time.
"""
from __future__ import annotations

from typing import Sequence


def partition_sources(costs: Sequence[float], world: int) -> list:
    """Greedy longest-processing-time partition; deterministic (ties by index)."""
    if world <= 0:
        raise ValueError("world must be positive")
    order = sorted(range(len(costs)), key=lambda a: (-float(costs[a]), a))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for a in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(a)
        load[r] += float(costs[a])
    return [sorted(p) for p in parts]


def source_cost(nodes: int, levels: int, rhs: int) -> float:
    return float(nodes) * float(rhs) * float(levels)


def reduce_model_gradient(g, group=None):
    """J^T y across ranks: in-place sum of each rank's partial sum over its sources."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return g
