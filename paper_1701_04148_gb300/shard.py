"""Assignment of independent sketches to ranks (one process per GPU).

A single SF-sketch does not shard: every update couples all d rows through the minimum over
rows (Sec. 3.4 insertion), so rows cannot live on different GPUs without two exchanges per
chunk.  Independent sketches -- the monitoring nodes of Sec. 1.1, or the Slims a collector
serves -- shard with no collective on the data path: each rank owns a disjoint subset and
processes it alone.  `assign` balances the ranks by total stream length (longest-processing-time
first); only host-side bookkeeping (gathering results, timing) crosses ranks.
"""
from __future__ import annotations

import heapq


def assign(lengths, world: int):
    """Rank of each sketch: greedy longest-first onto the least-loaded rank (deterministic)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(lengths)), key=lambda i: (-int(lengths[i]), i))
    heap = [(0, r) for r in range(world)]
    owner = [0] * len(lengths)
    for i in order:
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + int(lengths[i]), r))
    return owner


def owned(lengths, world: int, rank: int):
    """Indices of the sketches rank `rank` processes."""
    return [i for i, r in enumerate(assign(lengths, world)) if r == rank]


def imbalance(lengths, world: int) -> float:
    """max rank load / mean rank load of the assignment."""
    loads = [0] * world
    for i, r in enumerate(assign(lengths, world)):
        loads[r] += int(lengths[i])
    mean = sum(loads) / world
    return max(loads) / mean if mean else 1.0
