"""Host-side logic of multi-GPU runs: one process per GPU, each advancing its own
independently seeded problem (the path shards only as independent problems; there is no
data-path collective).  Timing is reduced as the maximum over ranks."""
from __future__ import annotations

import os


def env():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of the problem a rank advances: distinct per rank, identical to base at rank 0."""
    return base_seed + rank


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group (identity when not initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds_max
