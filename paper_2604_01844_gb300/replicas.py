"""Whole-job timing of independent replicas (one process per GPU, no data exchange): every
rank runs the same step on its own device; the job's time is the slowest rank's, and the job's
rate is the units all ranks processed over that time.  Works with any initialised
torch.distributed process group (NCCL on GPUs, gloo on CPU)."""
from __future__ import annotations

import torch


def world() -> int:
    import torch.distributed as dist

    return dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1


def slowest(ms: float, device=None) -> float:
    """The maximum of `ms` over all ranks (the value itself on a single process)."""
    if world() == 1:
        return float(ms)
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ms_slowest: float, n_ranks: int) -> float:
    """Units per second of the whole job: every rank processes `units_per_rank` per step."""
    return units_per_rank * n_ranks / (ms_slowest * 1e-3)
