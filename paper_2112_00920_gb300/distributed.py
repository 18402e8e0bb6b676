"""Sharding of the two-step sub-simulations over ranks (one GPU per rank).

The shifted sub-simulations of Eq. 9 are independent (Sec. II.B step 3),
so ranks share no data while they propagate; the one exchange the method
needs is the final average over shifts (step 4), formed here from per-rank
sums of dJ_m(t) = J_m(t) - J_m(0-) with one all-reduce.
"""
from __future__ import annotations

import numpy as np


def shard_ranges(costs, world: int):
    """Contiguous, cost-balanced blocks of sub-simulations: returns a list
    of (begin, end) per rank covering range(len(costs)).  costs[m] is the
    work of sub-simulation m (e.g. n_k * n_bands * n_pts * n_steps)."""
    costs = np.asarray(costs, dtype=np.float64)
    n = costs.size
    if world < 1:
        raise ValueError("world must be >= 1")
    if n == 0:
        return [(0, 0)] * world
    cum = np.concatenate([[0.0], np.cumsum(costs)])
    total = cum[-1]
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        b = int(np.searchsorted(cum, target, side="left"))
        # take the boundary closer to the target, never going backwards
        if b > 0 and abs(cum[b - 1] - target) <= abs(cum[min(b, n)] - target):
            b -= 1
        bounds.append(min(max(b, bounds[-1]), n))
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def two_step_average(dj_sum, n_local: int, group=None):
    """(1/N_H) sum over all ranks' sub-simulations of dJ_m(t).

    dj_sum: (n_t, 3) sum over this rank's sub-simulations of dJ_m;
    n_local: number of sub-simulations on this rank.  Uses
    torch.distributed.all_reduce (any backend) when a process group is
    initialised, else returns the local average."""
    import torch
    import torch.distributed as dist

    local = np.asarray(dj_sum, dtype=np.float64)
    if not (dist.is_available() and dist.is_initialized()):
        return local / max(n_local, 1)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    buf = torch.zeros(local.size + 1, dtype=torch.float64, device=dev)
    buf[:-1] = torch.from_numpy(local.reshape(-1)).to(dev)
    buf[-1] = float(n_local)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    out = buf.cpu().numpy()
    return out[:-1].reshape(local.shape) / out[-1]


def rank_world(group=None):
    """(rank, world size) of the process group, (0, 1) without one."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def run_sharded(costs, run_block, group=None):
    """The two-step scheme over ranks: this rank runs its cost-balanced block
    [begin, end) of the sub-simulations through run_block(begin, end), which
    returns the sum over the block of dJ_m(t) as an (n_t, 3) array, and the
    ranks then form the average over all sub-simulations (Eq. 9) with one
    all-reduce.  Returns (average dJ (n_t, 3), (begin, end))."""
    rank, world = rank_world(group)
    begin, end = shard_ranges(costs, world)[rank]
    dj_sum = run_block(begin, end)
    return two_step_average(dj_sum, end - begin, group), (begin, end)

