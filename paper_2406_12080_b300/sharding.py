"""Multi-GPU layout of the render path: views are sharded across ranks, the hierarchy is replicated.

Views are independent given the hierarchy, so rendering a camera set on N GPUs needs no exchange:
each rank renders its own share (`shard_views`).  Hierarchy optimisation (Sec. 5.1) updates the
interior nodes shared by all views; with views sharded across ranks it has exactly one exchange per
step, the sum of the per-rank node gradients, done here as one all-reduce over a flat bucket
(`allreduce_grads`).  One process per GPU; the process group is the caller's (NCCL on GPUs, gloo
on CPU).
"""
from __future__ import annotations

import numpy as np


def shard_views(cams, rank: int, world: int):
    """Contiguous share of `cams` for `rank`, balanced by pixel count; every camera in exactly one share.

    The split points are where the running pixel count crosses k/world of the total, so shares differ
    by at most one camera's pixels.  Returns (first index, list of cameras).
    """
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank out of range")
    px = np.array([c.width * c.height for c in cams], dtype=np.float64)
    if len(cams) == 0:
        return 0, []
    csum = np.concatenate([[0.0], np.cumsum(px)])
    total = csum[-1]
    # boundary k: first index whose prefix reaches k/world of the total
    bounds = [0] + [int(np.searchsorted(csum, total * k / world, side="left")) for k in range(1, world)] + [len(cams)]
    bounds = np.maximum.accumulate(np.minimum(bounds, len(cams)))
    lo, hi = int(bounds[rank]), int(bounds[rank + 1])
    return lo, list(cams[lo:hi])


def allreduce_grads(grads: dict, group=None) -> dict:
    """Sums the gradient tensors of every rank in place (one all-reduce over a flat bucket)."""
    import torch
    import torch.distributed as dist
    keys = sorted(grads)
    flat = torch.cat([grads[k].reshape(-1) for k in keys])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for k in keys:
        n = grads[k].numel()
        grads[k].copy_(flat[off:off + n].view_as(grads[k]))
        off += n
    return grads
