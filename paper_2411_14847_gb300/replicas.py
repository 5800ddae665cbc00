"""Host logic of running the timestep loop as independent replicas, one process per GPU.

The streaming reconstruction has no exchange step inside a timestep: each rank runs its own
scene's timesteps (replicas, weak scaling) and only the timing is combined -- the slowest rank's
elapsed time bounds the job, and the job's throughput counts every rank's timesteps.
"""
from __future__ import annotations

import torch


def replica_seed(base: int, rank: int) -> int:
    """Seed of a rank's synthetic scene (distinct per rank, reproducible)."""
    return int(base) + int(rank)


def max_over_ranks(ms: float, dist=None, device="cpu") -> float:
    """Largest value of ms over all ranks (ms itself without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def seconds_per_timestep(ms_max: float, steps: int, world: int) -> float:
    """Whole-job seconds per timestep: world * steps timesteps finished within ms_max."""
    return ms_max / 1e3 / (steps * world)
