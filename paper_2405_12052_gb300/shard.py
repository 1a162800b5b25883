"""Host side of the sharded step: the exchange between processes.

The library computes each shard's exact column totals and the update from
the gathered totals (km_shard_totals, km_shard_update in include/km.h); this
module moves the small tables between ranks with torch.distributed (gloo on
host tensors, or NCCL on device tensors): one max-reduction of the grid
exponent at set-up, one all-gather of K*(d+1) int128 values per step.  The
gathered tables are kept in rank order, the order km_shard_update adds them.
"""
from __future__ import annotations

import numpy as np


def common_grid_exponent(g, dist, group=None) -> int:
    """Every shard's grid exponent, reduced to the maximum, set on `g`."""
    import torch
    t = torch.tensor([g.grid_exponent()], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    ex = int(t.item())
    g.set_grid_exponent(ex)
    return ex


def gather_totals(totals: np.ndarray, dist, group=None) -> np.ndarray:
    """All-gather one (K*(d+1), 2) int64 table per rank: (ranks, K*(d+1), 2)
    in rank order on every rank."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(totals, dtype=np.int64))
    out = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(out, t, group=group)
    return np.stack([o.numpy() for o in out])


def sharded_step(g, dist, group=None) -> None:
    """One step of a sharded context: assign, exchange, update."""
    g.assign_async()
    g.shard_update(gather_totals(g.shard_totals(), dist, group))
