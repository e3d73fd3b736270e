"""Work split across ranks (one process per GPU).

Shots are independent problems, so the only data exchanged between ranks is the
sum of the misfit gradients of a multi-shot job: every rank takes every
world-th shot, sums its shots' misfits and fp64 gradients, and one all-reduce
(SUM) adds the ranks' partial sums.  Timing takes the maximum over ranks.  With
one rank (or no process group) nothing is communicated.
"""
from __future__ import annotations

from typing import Callable, Sequence

import torch


def _group_size():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def my_shots(n_shots: int, rank: int, world: int) -> list:
    """Indices of the shots rank `rank` of `world` runs: rank, rank + world, ..."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    return list(range(rank, n_shots, world))


def gradient_sum(shot_fn: Callable[[int], tuple], n_shots: int, like: torch.Tensor):
    """Misfit and fp64 gradient summed over `n_shots` shots split across ranks.

    shot_fn(i) returns (J_i, grad_i) for shot i (grad_i an fp64 tensor shaped
    like `like`, on its device).  Returns (J, grad) on every rank."""
    rank, world = _group_size()
    total = torch.zeros_like(like, dtype=torch.float64)
    J = 0.0
    for i in my_shots(n_shots, rank, world):
        Ji, gi = shot_fn(i)
        J += float(Ji)
        total += gi
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(total, op=dist.ReduceOp.SUM)
        Jt = torch.tensor([J], dtype=torch.float64, device=total.device)
        dist.all_reduce(Jt, op=dist.ReduceOp.SUM)
        J = float(Jt.item())
    return J, total


def max_over_ranks(x: float, device=None) -> float:
    """The maximum of a per-rank number (a timing) over all ranks."""
    rank, world = _group_size()
    if world == 1:
        return float(x)
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: Sequence[float] | float, seconds_max: float, world: int = 1) -> float:
    """Whole-job throughput: the units all ranks processed divided by the
    slowest rank's time."""
    units = sum(units_per_rank) if isinstance(units_per_rank, (list, tuple)) else units_per_rank * world
    return float(units) / float(seconds_max)
