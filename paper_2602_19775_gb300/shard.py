"""Trajectory sharding across ranks (one process per GPU).

Trajectories are independent and every random number of trajectory i comes from Philox counters keyed by
its global id, so splitting the trajectory ids into contiguous ranges changes no result: rank r simulates
global ids [offset_r, offset_r + count_r) by passing traj_offset = offset_r. A loss on ensemble means
couples the ranks through two small all-reduces per step: the per-sample sums of the observables before
the loss, and the parameter gradient after the backward. These helpers hold that host logic; the
simulation itself runs in the library on each rank's GPU.
"""
from __future__ import annotations

import torch


def shard_range(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous share of n_total trajectory ids for `rank`: (offset, count); the first n_total % world
    ranks take one more."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_total, world)
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def global_ensemble_mean(local_obs: torch.Tensor) -> torch.Tensor:
    """Mean over all ranks' trajectories of obs [n_local, ...] (float64 sums, one all-reduce of
    [prod(shape[1:]) + 1] values)."""
    flat = local_obs.reshape(local_obs.shape[0], -1).to(torch.float64)
    buf = torch.cat([flat.sum(0), torch.tensor([float(flat.shape[0])], dtype=torch.float64, device=flat.device)])
    dist = _dist()
    if dist is not None:
        dist.all_reduce(buf)
    return (buf[:-1] / buf[-1]).reshape(local_obs.shape[1:])


def global_gradient(local_dtheta: torch.Tensor) -> torch.Tensor:
    """Sum of the ranks' parameter gradients (one all-reduce of P values)."""
    g = local_dtheta.clone()
    dist = _dist()
    if dist is not None:
        dist.all_reduce(g)
    return g


def max_over_ranks(seconds: float, device=None) -> float:
    """Largest wall time over the ranks (the time of the whole job)."""
    dist = _dist()
    if dist is None:
        return seconds
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def total_over_ranks(count: int, device=None) -> int:
    """Sum of an integer count (e.g. SSA steps) over the ranks."""
    dist = _dist()
    if dist is None:
        return count
    t = torch.tensor([count], dtype=torch.int64, device=device)
    dist.all_reduce(t)
    return int(t.item())
