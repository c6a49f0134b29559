"""Placement of independent graphs on several GPUs (one process per GPU).

A batch of DAGs shards without any exchange: every graph is partitioned on one GPU, alone. The
graphs go to the ranks by longest-processing-time-first list scheduling (Graham, 1969) with the edge
count as the work estimate: heaviest graph first, each to the rank with the least work so far. It
keeps the largest rank load within 4/3 of the best possible, and it is deterministic, so every rank
computes the same placement without communicating.
"""
from __future__ import annotations

import heapq


def lpt(weights, parts: int):
    """Indices of `weights` per part: items in (weight desc, index asc) order, each to the part with
    the least load (lowest part index on ties).  Each list is ascending."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-int(weights[i]), i))
    heap = [(0, p) for p in range(parts)]
    out = [[] for _ in range(parts)]
    for i in order:
        load, p = heapq.heappop(heap)
        out[p].append(i)
        heapq.heappush(heap, (load + int(weights[i]), p))
    return [sorted(x) for x in out]
