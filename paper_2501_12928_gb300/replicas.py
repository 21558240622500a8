"""Replicas across GPUs: independent prior points, one process per GPU.

The batch of prior points shards across ranks with no exchange of matrices
(each rank holds its own precompute); the only communication is a gather of
the per-point results (lnL and status) to every rank and the maximum of the
per-rank times.  Works with the gloo (CPU) and nccl backends of
torch.distributed.
"""

from __future__ import annotations

import numpy as np


def shard_bounds(n: int, rank: int, world: int):
    """Contiguous [lo, hi) slice of n points for `rank` (sizes differ by at most one)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def evaluate_sharded(loglike, phi, group=None):
    """Evaluate loglike on this rank's shard of phi and gather every rank's
    values, in the original order, to every rank.  loglike returns
    (lnl, status) arrays for its shard."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    phi = np.asarray(phi, np.float64)
    lo, hi = shard_bounds(len(phi), rank, world)
    lnl, st = loglike(phi[lo:hi]) if hi > lo else (np.zeros(0), np.zeros(0, np.int32))
    width = max(shard_bounds(len(phi), r, world)[1] - shard_bounds(len(phi), r, world)[0] for r in range(world))
    dev = torch.device("cuda") if dist.get_backend(group) == "nccl" else torch.device("cpu")
    buf = torch.full((width, 2), float("nan"), dtype=torch.float64, device=dev)
    buf[: hi - lo, 0] = torch.as_tensor(np.asarray(lnl, np.float64))
    buf[: hi - lo, 1] = torch.as_tensor(np.asarray(st, np.float64))
    out = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(out, buf, group=group)
    vals = np.empty(len(phi))
    stat = np.empty(len(phi), np.int32)
    for r in range(world):
        a, b = shard_bounds(len(phi), r, world)
        o = out[r].cpu().numpy()
        vals[a:b] = o[: b - a, 0]
        stat[a:b] = o[: b - a, 1].astype(np.int32)
    return vals, stat


def max_over_ranks(x: float, group=None) -> float:
    """The maximum of a per-rank number (e.g. elapsed seconds)."""
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda") if dist.get_backend(group) == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
