"""Whole-job throughput over replica ranks (one independent system per GPU).

The solver path has no collective: under torchrun every rank solves its own
augmented system.  The only cross-rank steps are a barrier around the timed
region and the reduction that turns per-rank times into a whole-job number.
"""
from __future__ import annotations


def job_throughput(local_seconds: float, units_per_rank: int, world: int, device=None) -> float:
    """Units of all ranks divided by the slowest rank's time (MAX over ranks).

    With world == 1 no process group is needed.  Otherwise a process group
    must be initialised (gloo on CPU, NCCL on GPUs; ``device`` selects where
    the scalar lives).
    """
    t = float(local_seconds)
    if world > 1:
        import torch
        import torch.distributed as dist
        buf = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(buf, op=dist.ReduceOp.MAX)
        t = float(buf.item())
    if t <= 0:
        raise ValueError("non-positive time")
    return world * units_per_rank / t


def rank_seed(base: int, rank: int) -> int:
    """Seed of the system a rank solves (rank 0 keeps the workload's own seed)."""
    return base if rank == 0 else base + 17 * rank
