"""Replica bookkeeping for multi-GPU runs (one process per GPU, torchrun env).

The solver itself has no collective: every rank solves its own independent
systems (weak scaling).  Ranks only agree on timing: a barrier on both sides
of the timed region and the maximum step time over ranks; the whole-job
throughput is all ranks' units divided by that time.  Works with the NCCL
(CUDA tensors) and gloo (CPU tensors) backends."""
from __future__ import annotations

import os


def env():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def job_throughput(units_per_rank: float, step_s_per_rank: float, device=None) -> float:
    """Whole-job units/s: every rank's units over the slowest rank's time."""
    import torch.distributed as dist
    n = dist.get_world_size() if (dist.is_available() and dist.is_initialized()) else 1
    slowest = max_over_ranks(step_s_per_rank, device)
    return n * units_per_rank / slowest
