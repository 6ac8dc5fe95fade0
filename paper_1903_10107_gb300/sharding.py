"""Frame sharding across GPUs.

Reconciliation frames are independent, so N GPUs each decode their own share
and nothing is exchanged on the data path.  Two layouts:

* weak scaling: every rank decodes ``per_rank`` frames of its own, frames
  ``[rank * per_rank, (rank + 1) * per_rank)`` of the seeded stream;
* strong scaling: ``total`` frames split into contiguous, near-equal shares.

After a timed region the ranks agree on the job's time (the maximum over
ranks) and totals (sums over ranks) with one all-reduce each.
"""
from __future__ import annotations

import numpy as np


def weak_shard(per_rank: int, rank: int, world: int):
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return rank * per_rank, per_rank


def strong_shard(total: int, rank: int, world: int):
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    base, extra = divmod(total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def reduce_max_sum(values_max, values_sum, dist=None, device=None):
    """(max over ranks of values_max, sum over ranks of values_sum) as numpy
    float64 arrays; with ``dist`` None (one process) the inputs come back."""
    vm = np.asarray(values_max, dtype=np.float64)
    vs = np.asarray(values_sum, dtype=np.float64)
    if dist is None:
        return vm, vs
    import torch
    tm = torch.from_numpy(vm.copy())
    ts = torch.from_numpy(vs.copy())
    if device is not None:
        tm, ts = tm.to(device), ts.to(device)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    dist.all_reduce(ts, op=dist.ReduceOp.SUM)
    return tm.cpu().numpy(), ts.cpu().numpy()
