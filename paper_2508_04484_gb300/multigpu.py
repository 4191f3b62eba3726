"""Several GPUs, one process each: beams are independent low-rank states (no exchange while
stepping), so a multi-beam plan is split by beam and the only collective is the final sum of
the deposited energy over ranks. One beam on several GPUs (spatial decomposition with halo
exchange and Gram all-reduce) is not implemented.

torch.distributed is plumbing here: the dose lives in a torch tensor (CUDA with NCCL, or CPU
with gloo for the host-side tests).
"""
from __future__ import annotations


def shard_beams(beams, rank: int, world: int):
    """Beams of this rank: round-robin over the plan, so that every beam is solved once."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of {world}")
    return [b for i, b in enumerate(beams) if i % world == rank]


def shard_indices(n_beams: int, rank: int, world: int):
    return [i for i in range(n_beams) if i % world == rank]


def reduce_dose(dose, group=None):
    """Sum the per-rank deposits in place on every rank (the plan's total dose)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(dose, op=dist.ReduceOp.SUM, group=group)
    return dose


def max_over_ranks(value: float, device="cpu", group=None) -> float:
    """The slowest rank's time (the job ends when the last rank does)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
