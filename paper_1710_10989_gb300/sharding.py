"""Partition of a batch of independent exp(A) problems across ranks.

Matrices are independent, so a multi-GPU run needs no data-path collective:
each rank takes a shard and runs the batched launch on it. Shards are built
by longest-processing-time-first greedy assignment on the cost of each
exp(A): N^3 (pi_m + s), the number of dense products (Table 3's pi_m for the
degree plus s squarings, the paper's cost unit) times the N^3 of each one.
Without the (m, s) term a batch whose norms span 1e-3 .. 1e2 (3 to 12
products per matrix) can leave one shard several times heavier than another
at equal N^3; with it the largest shard stays within a few percent of the
mean for batches of thousands of uneven matrices.
"""
from __future__ import annotations

import heapq


def costs_of(sizes, products=None) -> list[int]:
    """N^3 (pi_m + s) per matrix; `products` (pi_m + s per matrix) defaults to 1."""
    if products is None:
        return [int(n) ** 3 for n in sizes]
    if len(products) != len(sizes):
        raise ValueError("one product count per matrix")
    return [int(n) ** 3 * max(1, int(p)) for n, p in zip(sizes, products)]


def shard_indices(sizes, rank: int, world: int, products=None) -> list[int]:
    """Indices of `sizes` assigned to `rank` (deterministic on every rank).
    `products[i]` = pi_m + s of matrix i (its (m, s) from the theta rule)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    cost = costs_of(sizes, products)
    order = sorted(range(len(sizes)), key=lambda i: (-cost[i], i))
    heap = [(0, r) for r in range(world)]
    mine = []
    for i in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(i)
        heapq.heappush(heap, (load + cost[i], r))
    return mine


def shard_costs(sizes, world: int, products=None) -> list[int]:
    cost = costs_of(sizes, products)
    return [sum(cost[i] for i in shard_indices(sizes, r, world, products)) for r in range(world)]
