"""Host-side logic of multi-GPU runs: one process per GPU (torchrun), no data-path collective.

The batched workload is a set of independent 1D problems (each with its own grid, boundary
conditions, Lax-Friedrichs constants and CFL step), so it shards by problem: every rank
advances its share through its own weno_theta_step_batched call and no state crosses ranks.
The share is a longest-processing-time-first (LPT) partition on the cell counts: problems
sorted by length, largest first, each given to the rank with the fewest cells so far, which
keeps the ranks' cell totals within the largest problem of each other.  The only collectives
are the timing barrier and the maximum of the per-rank times.
"""
from __future__ import annotations

import heapq
import os

import numpy as np


def env():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def lpt_partition(lengths, world: int):
    """Problem indices of each rank: problems by decreasing length (ties by index), each to the
    rank holding the fewest cells so far (ties to the lowest rank).  Deterministic, so every
    rank computes the same partition from the same lengths.  Each rank's indices are returned
    in the order they were assigned (largest first)."""
    lengths = np.asarray(lengths, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(lengths)), key=lambda p: (-int(lengths[p]), p))
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for p in order:
        load, r = heapq.heappop(heap)
        parts[r].append(p)
        heapq.heappush(heap, (load + int(lengths[p]), r))
    return [np.asarray(x, dtype=np.int64) for x in parts]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group (identity when not initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a per-rank float over the default process group (identity when not initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_all_ranks: float, seconds_max: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_all_ranks / seconds_max
