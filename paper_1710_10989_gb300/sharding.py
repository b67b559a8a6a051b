"""Partition of a batch of independent exp(A) problems across ranks.

Matrices are independent, so a multi-GPU run needs no data-path collective:
each rank takes a shard and runs the batched launch on it. Shards are built
by longest-processing-time-first greedy assignment on the cost N^3 (the
products dominate and each costs 2 N^3), which keeps the largest shard within
a few percent of the mean for batches of thousands of uneven matrices.
"""
from __future__ import annotations

import heapq


def shard_indices(sizes, rank: int, world: int) -> list[int]:
    """Indices of `sizes` assigned to `rank` (deterministic on every rank)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    heap = [(0, r) for r in range(world)]
    mine = []
    for i in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(i)
        heapq.heappush(heap, (load + int(sizes[i]) ** 3, r))
    return mine


def shard_costs(sizes, world: int) -> list[int]:
    return [sum(int(sizes[i]) ** 3 for i in shard_indices(sizes, r, world)) for r in range(world)]
