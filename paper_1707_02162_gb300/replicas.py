"""Host-side logic for running independent REDO replicas on several GPUs.

Pulses, noise realisations and GRAPE instances are independent, so a job
shards by giving every rank its own batch (no collective on the data path);
the only communication is the timing reduction: the job's time is the
slowest rank's, and its throughput counts the units of all ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s batch; rank 0 keeps the base seed."""
    return base_seed if rank == 0 else base_seed + 7919 * rank


def aggregate_throughput(units_per_rank: float, local_seconds: float, group=None) -> tuple[float, float]:
    """(job throughput, job seconds): units of all ranks over the max-over-ranks time."""
    if not (dist.is_available() and dist.is_initialized()):
        return units_per_rank / local_seconds, local_seconds
    t = torch.tensor([local_seconds], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    world = dist.get_world_size(group)
    slowest = float(t.item())
    return world * units_per_rank / slowest, slowest
