"""Host-side logic for running the library on several GPUs of one node, one process per
GPU (torch.distributed; NCCL on GPUs, gloo on CPU for tests).

A single stream does not shard: its rows are sequential (each row's rank decision
depends on every earlier row, Algorithm 1), so N processes run N independent replicas
and no data-path collective exists. Independent streams of a batch shard by instance:
each rank takes a subset chosen by longest-processing-time-first on the cost
n_b * m_b * min(n_b, r_b) (the O(mr) work per row of Algorithm 1 over n_b rows), runs it
in its own persistent kernel, and only host-side results are gathered.
"""
from __future__ import annotations

import heapq

import numpy as np


def instance_cost(n, m, r) -> np.ndarray:
    """Work estimate per instance: rows x columns x rank bound (O(mr) per row)."""
    n = np.asarray(n, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    return n * m * np.minimum(n, r)


def lpt_partition(costs, world_size: int) -> list:
    """Longest-processing-time-first partition of instances over ranks.

    Instances are taken in decreasing cost (ties by index) and each goes to the rank with
    the least load so far (ties by rank). Returns one sorted index array per rank; the
    arrays partition range(len(costs)). Deterministic, so every rank computes the same
    partition without communicating."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, rk) for rk in range(world_size)]
    parts = [[] for _ in range(world_size)]
    for i in order:
        load, rk = heapq.heappop(heap)
        parts[rk].append(i)
        heapq.heappush(heap, (load + costs[i], rk))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (the whole job's time is the slowest
    rank's). Returns the value unchanged when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a per-rank scalar over all ranks (units processed by the whole job)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_this_rank: float, ms_this_rank: float, device=None) -> tuple:
    """Whole-job throughput: units processed by all ranks / the slowest rank's time.
    Returns (units per second, max milliseconds, total units)."""
    ms = max_over_ranks(ms_this_rank, device)
    units = sum_over_ranks(units_this_rank, device)
    return units / (ms / 1e3), ms, units
