"""Host logic for running independent replicas on several GPUs.

A single chain has a serial accept-by-accept dependency and does not shard, so
the only multi-GPU form of the method is independent replicas: independent
chains (batch) or requests (serving) partitioned across ranks, each rank on its
own GPU, and the slowest rank's time as the job's time.  No collective is
needed on the data path; torch.distributed (NCCL on GPUs, gloo on CPUs) only
reduces the per-rank times.
"""
from __future__ import annotations

import heapq
from typing import Sequence


def chain_cost(N: int, iters: int, accept_rate: float = 0.01) -> float:
    """Estimated work of a chain: proposals plus accepted swaps times their O(N^2) update."""
    return float(iters) * (1.0 + accept_rate * N * N / 64.0)


def partition_by_cost(costs: Sequence[float], world: int) -> list[list[int]]:
    """Longest-processing-time-first assignment of items to `world` ranks.

    Returns one list of item indices per rank; every item appears exactly once,
    and the heaviest rank carries at most 4/3 of the optimum (Graham's bound).
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0.0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return parts


def stream_id_for(rank: int, base: int = 0) -> int:
    """Philox stream (counter word 2) of a replica: distinct per rank."""
    return base + rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (the job's time); identity without dist."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
