"""Host-side logic for running the many-graph form on several GPUs (one process per GPU).

Graphs are independent units: each rank takes a share of them and runs its own
arena and batch; the only cross-rank communication is the timing reduction
(max over ranks) and the result gather, both on the host side of the job.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence


def lpt_partition(weights: Sequence[float], world: int) -> List[List[int]]:
    """Greedy largest-first bin packing: item indices per rank, balancing the sum of weights.

    Deterministic (ties by index), so every rank computes the same partition independently.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-float(weights[i]), i))
    heap = [(0.0, r) for r in range(world)]
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(weights[i]), r))
    for p in parts:
        p.sort()
    return parts


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of a per-rank float across the process group (identity without one)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
