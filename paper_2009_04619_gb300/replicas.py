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


def gradient_sum(shot_fn: Callable, n_shots: int, like: torch.Tensor, workers: int = 1,
                 streams: Sequence | None = None):
    """Misfit and fp64 gradient summed over `n_shots` shots split across ranks.

    shot_fn(i, k) returns (J_i, grad_i) for shot i computed by worker k (grad_i
    an fp64 tensor shaped like `like`, on its device, valid until that worker's
    next call).  With workers > 1 each worker is a host thread (the library
    releases the GIL while a shot runs), inside streams[k] when given, so the
    shots' kernels overlap on the GPU.  Shot i goes to worker i mod workers and
    every worker sums its shots in order, so the result does not depend on
    timing.  Returns (J, grad) on every rank."""
    import threading

    rank, world = _group_size()
    mine = my_shots(n_shots, rank, world)
    parts = [mine[k::workers] for k in range(workers)]
    totals = [None] * workers
    Js = [0.0] * workers
    errors = []

    def run(k):
        try:
            ctx = torch.cuda.stream(streams[k]) if streams is not None else _nullcontext()
            with ctx:  # the sum lives on the worker's stream, like its shots
                totals[k] = torch.zeros_like(like, dtype=torch.float64)
                for i in parts[k]:
                    Ji, gi = shot_fn(i, k)
                    Js[k] += float(Ji)
                    totals[k] += gi
        except BaseException as e:  # re-raised in the caller's thread
            errors.append(e)

    if workers == 1:
        run(0)
    else:
        threads = [threading.Thread(target=run, args=(k,)) for k in range(workers)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
    if errors:
        raise errors[0]
    if streams is not None:
        torch.cuda.synchronize()
    total = totals[0]
    for t in totals[1:]:
        total += t
    J = sum(Js)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(total, op=dist.ReduceOp.SUM)
        Jt = torch.tensor([J], dtype=torch.float64, device=total.device)
        dist.all_reduce(Jt, op=dist.ReduceOp.SUM)
        J = float(Jt.item())
    return J, total


class _nullcontext:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


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
