"""Sharding the receivers of one scene over several ranks (torch.distributed).

Each rank evaluates the received power of its own contiguous block of
receivers; the loss -min_r P_r needs one exchange, a MINLOC reduction of the
ranks' (min power, global index) pairs with ties to the lowest index, and
the gradient needs one more, a sum of the ranks' gradients (only the rank
that owns the argmin has a non-zero one).  Works with any backend (gloo on
CPU, NCCL on GPUs).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(n: int, world: int, rank: int) -> tuple[int, int]:
    """[start, stop) of rank's block when n items are split as evenly as possible."""
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def minloc_allreduce(value: float, index: int, group=None) -> tuple[float, int]:
    """Global (min value, its index) over the ranks; ties go to the lowest index.
    A rank with nothing to offer passes value = +inf."""
    world = dist.get_world_size(group)
    mine = torch.tensor([float(value), float(index)], dtype=torch.float64)
    parts = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    best = min(((float(p[0]), int(p[1])) for p in parts), key=lambda t: (t[0], t[1]))
    return best


def sharded_min_loss(power_local, start: int, group=None) -> tuple[float, int]:
    """(loss, global argmin) of -min over all ranks' receivers; power_local is this
    rank's block (any array-like), whose first receiver has global index start."""
    p = torch.as_tensor(power_local, dtype=torch.float64).reshape(-1)
    if p.numel():
        i = int(torch.argmin(p))           # first minimum within the block
        v, idx = float(p[i]), start + i
    else:
        v, idx = float("inf"), 2 ** 52
    best, arg = minloc_allreduce(v, idx, group)
    return -best, arg


def sum_allreduce(t: torch.Tensor, group=None) -> torch.Tensor:
    t = t.clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t
