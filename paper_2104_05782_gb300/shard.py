"""Host-side sharding of independent factorizations across processes / GPUs.

A single factorization does not shard (the block steps form a chain with a
panel dependency every b columns), so N GPUs run N independent replicas.  A
batch of independent matrices does shard: each rank takes a longest-
processing-time-first share of the estimated flops and factors it on its own
GPU; no data-path collective is needed, only a max over ranks of the elapsed
time.
"""
from __future__ import annotations

import heapq


def lpt_partition(costs, world: int):
    """Indices of `costs` split over `world` ranks, longest first onto the least
    loaded rank (ties: lowest rank).  Deterministic; every rank computes the
    same partition from the same costs.  Makespan <= (4/3 - 1/(3 world)) x optimum."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def loads(costs, parts):
    return [sum(costs[i] for i in p) for p in parts]
