"""Sharding independent samples across ranks (one process per GPU).

The batched porous configuration is a set of independent samples: a sample's
time steps read only its own nodes, so ranks split the samples between them
and exchange nothing while stepping.  Two splits:

* strong: one fixed set of samples divided among the ranks, balanced by node
  count (longest-processing-time greedy: samples in decreasing node count,
  each to the rank with the fewest nodes so far; ties to the lower rank and
  the lower sample index, so every rank computes the same assignment);
* weak: every rank owns a full set of its own (seeds offset by the rank), so
  the work per GPU stays fixed as ranks are added.

Per-sample results (steps, permeability) come back to rank 0 in the original
sample order with merge_by_sample().
"""
from __future__ import annotations

import heapq


def assign_balanced(weights, world: int) -> list:
    """Split sample indices 0..len(weights)-1 among `world` ranks by the
    greedy longest-processing-time rule.  Returns one sorted index list per
    rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-int(weights[i]), i))
    heap = [(0, r) for r in range(world)]
    heapq.heapify(heap)
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(weights[i]), r))
    return [sorted(v) for v in out]


def rank_seed_offset(rank: int, samples_per_rank: int) -> int:
    """Weak scaling: rank r's samples use seeds offset by r * samples_per_rank."""
    return int(rank) * int(samples_per_rank)


def merge_by_sample(per_rank: list, assignment: list, n_samples: int) -> list:
    """per_rank[r] lists rank r's per-sample results in the order of
    assignment[r]; returns them as one list in sample order."""
    out = [None] * n_samples
    for vals, idx in zip(per_rank, assignment):
        if len(vals) != len(idx):
            raise ValueError("a rank returned the wrong number of results")
        for v, i in zip(vals, idx):
            out[i] = v
    if any(v is None for v in out):
        raise ValueError("a sample has no result")
    return out


def imbalance(weights, assignment) -> float:
    """Largest rank load over the mean load (1 = perfect balance)."""
    loads = [sum(int(weights[i]) for i in idx) for idx in assignment]
    mean = sum(loads) / len(loads)
    return max(loads) / mean if mean > 0 else 1.0
