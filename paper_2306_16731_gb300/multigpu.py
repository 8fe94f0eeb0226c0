"""Host-side logic for running the batched update on several GPUs.

Patches are independent given their halos and each carries its own time
step (local time stepping, arXiv:2306.16731 Sec. 2.2), so a batch shards
across ranks with no exchange during a step: each rank advances its own
contiguous range of patches.  The only collective work is bookkeeping
around the timed region (a barrier and a maximum of the per-rank times),
which runs on whatever ``torch.distributed`` backend is initialised (NCCL on
GPUs, gloo on CPUs for the tests).
"""
from __future__ import annotations

import numpy as np


def shard_patches(patch_size, dim: int, world: int, rank: int):
    """Contiguous range [begin, end) of patches for ``rank`` such that the
    ranges cover all patches once and each holds about the same number of
    interior volumes (sum of p_i^dim)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    p = np.asarray(patch_size, dtype=np.int64).reshape(-1)
    work = np.concatenate([[0], np.cumsum(p ** dim)])
    total = work[-1]
    # rank r starts at the first patch whose preceding work reaches r/world of the total
    targets = [total * r / world for r in range(world + 1)]
    cuts = [int(np.searchsorted(work, t, side="left")) for t in targets]
    cuts[0], cuts[-1] = 0, len(p)
    for r in range(1, world + 1):            # keep the cuts monotone
        cuts[r] = max(cuts[r], cuts[r - 1])
    return cuts[rank], cuts[rank + 1]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity without a
    process group)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds_max: float, dist=None, device=None) -> float:
    """Units processed by all ranks divided by the slowest rank's time."""
    total = float(units_per_rank)
    if dist is not None and dist.is_available() and dist.is_initialized():
        import torch
        t = torch.tensor([total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        total = float(t.item())
    return total / seconds_max
