"""Splitting independent problems of a batched solve across ranks (one GPU
per rank, no data exchange): longest-processing-time-first on an estimated
cost, so every rank gets about the same work.  The cost of a problem is its
points times its step count; for a CFL-limited explicit scheme the step count
grows like the nodes per axis, so points^(1 + 1/d) is used when the step
count is not known."""
from __future__ import annotations

import heapq


def estimated_cost(spec: dict) -> float:
    pts = 1
    for v in spec["n"]:
        pts *= int(v)
    return float(pts) ** (1.0 + 1.0 / spec["ndim"])


def shard(costs, world: int):
    """Indices of the problems each of `world` ranks solves (a partition of
    range(len(costs))), greedy: the costliest unassigned problem goes to the
    least loaded rank.  Deterministic, so every rank computes the same split."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(v) for v in out]
