"""Shot parallelism across ranks (one process per GPU).

Shots are independent: each rank models its own shots, so forward modelling
needs no communication at all.  The FWI gradient is the sum over shots, so the
only exchange is one all-reduce of the per-rank gradient sums, done in float64
(the paper's closing remark on running inversion operators in parallel across
processes, Sec. 6).
"""
from __future__ import annotations


def shard(nshots: int, rank: int, world: int) -> list:
    """Shot indices of `rank`: round-robin over ranks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    return list(range(rank, nshots, world))


def allreduce_gradient(grad, group=None):
    """Sum a per-rank gradient (torch tensor) over all ranks in float64, in
    place of the caller's dtype; returns the summed tensor (float64)."""
    import torch
    import torch.distributed as dist
    g = grad.to(torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return g
