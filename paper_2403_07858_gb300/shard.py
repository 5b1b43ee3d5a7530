"""Splitting one count across GPUs (or processes) by search-tree roots.

Roots' search trees share nothing (Sec. III-B), so a count splits into
disjoint root ranges with no exchange during the search; the only collective
is one exact 128-bit sum at the end.  Host logic only: each rank counts its
range with ``Graph.count_ex(..., roots=...)`` on its own GPU.
"""
from __future__ import annotations

import numpy as np


def root_ranges(weights, world: int) -> list[tuple[int, int]]:
    """Contiguous ranges of roots, one per rank, with near-equal total weight
    (weights: a per-root work estimate, e.g. the degree of each anchor vertex
    squared).  Every root is in exactly one range; ranges may be empty."""
    w = np.asarray(weights, dtype=np.float64)
    n = w.size
    if world < 1:
        raise ValueError("world must be >= 1")
    cum = np.cumsum(w)
    total = float(cum[-1]) if n else 0.0
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(cum, total * r / world, side="right")) if total > 0 else (n * r) // world)
    cuts.append(n)
    cuts = np.maximum.accumulate(np.clip(cuts, 0, n)).tolist()
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]


def allreduce_u128(value: int, group=None) -> int:
    """Exact sum of a non-negative integer below 2^128 over all ranks.

    The value travels as four 32-bit limbs in int64 (sums of up to 2^31 ranks
    cannot overflow), carries are resolved after the reduction, and a total at
    or above 2^128 raises OverflowError."""
    import torch
    import torch.distributed as dist
    if not 0 <= value < 1 << 128:
        raise ValueError("value outside [0, 2^128)")
    limbs = [(value >> (32 * i)) & 0xFFFFFFFF for i in range(4)]
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor(limbs, dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    total = sum(int(x) << (32 * i) for i, x in enumerate(t.tolist()))
    if total >= 1 << 128:
        raise OverflowError("sum exceeds 2^128 - 1")
    return total


def count_sharded(graph, p: int, q: int, anchor: str, rank: int, world: int, weights, group=None) -> int:
    """This rank's share of the (p,q) count, summed over all ranks."""
    r0, r1 = root_ranges(weights, world)[rank]
    mine = graph.count_ex(p, q, anchor=anchor, roots=(r0, r1))[0] if r1 > r0 else 0
    return allreduce_u128(mine, group)
