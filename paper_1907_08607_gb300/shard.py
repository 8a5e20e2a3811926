"""Splitting the counting of one graph over processes or devices (host logic).

The outer loop of Algorithm 2 runs over independent owners, so a graph can be
cut into owner ranges, each range counted on its own (pb_count_owner_range)
and the partial counts added element by element.  `partition` chooses ranges
of nearly equal wedge mass from the per-owner wedge prefix; `sum_parts` adds
the parts across a torch.distributed process group (wrapping uint64 addition,
carried in int64 tensors).
"""
from __future__ import annotations

import numpy as np


def partition(prefix, k: int) -> list[tuple[int, int]]:
    """k contiguous ranges [lo, hi) covering [0, n) whose wedge masses are as
    equal as owner granularity allows; prefix is the exclusive prefix (n + 1
    entries, prefix[n] = W)."""
    prefix = np.asarray(prefix, dtype=np.uint64)
    n = prefix.shape[0] - 1
    if k < 1:
        raise ValueError("k must be positive")
    total = int(prefix[-1])
    cuts = [0]
    for i in range(1, k):
        target = np.uint64((total * i) // k)
        c = int(np.searchsorted(prefix, target, side="left"))
        cuts.append(min(max(c, cuts[-1]), n))
    cuts.append(n)
    return [(cuts[i], cuts[i + 1]) for i in range(k)]


def sum_parts(tensors, group=None):
    """All-reduce (sum) every tensor in place across the process group."""
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


def count_shard(graph, rank: int, world: int, agg: str = "auto", **kw):
    """Partial counts of this process's owner range (device tensors)."""
    lo, hi = partition(graph.wedge_prefix(), world)[rank]
    return graph.count_all(agg, owners=(lo, hi), on_device=True, **kw)
