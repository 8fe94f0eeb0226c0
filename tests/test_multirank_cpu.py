"""Multi-rank host logic on CPU with the gloo backend (world size 2).

The batched update shards across ranks without any exchange during a step;
what the ranks share is the bookkeeping around the timed region.  These
tests run real torch.distributed process groups on the CPU.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

from paper_2306_16731_gb300.multigpu import shard_patches


def test_shards_cover_every_patch_once_and_balance_volumes():
    from paper_2306_16731_gb300 import inputs
    w = inputs.config(4, num_patches=5000)
    for world in (1, 2, 3, 4, 8):
        ranges = [shard_patches(w.patch_size, 2, world, r) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == w.num_patches
        for (a, b), (c, d) in zip(ranges, ranges[1:]):
            assert b == c and a <= b
        work = [int(np.sum(w.patch_size[a:b].astype(np.int64) ** 2)) for a, b in ranges]
        assert max(work) - min(work) <= 2 * 32 * 32     # each cut is off by less than one largest patch
        assert sum(work) == w.interior_volumes


def test_shard_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard_patches([4, 4], 2, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2306_16731_gb300.multigpu import max_over_ranks, shard_patches, whole_job_rate
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [16] * 10 + [8] * 6
    a, b = shard_patches(sizes, 2, world, rank)
    my_vols = sum(s * s for s in sizes[a:b])
    my_time = 0.5 + rank            # the slowest rank decides
    tmax = max_over_ranks(my_time, dist)
    rate = whole_job_rate(my_vols, tmax, dist)
    dist.barrier()
    out[rank] = (a, b, tmax, rate)
    dist.destroy_process_group()


def test_two_rank_timing_and_aggregation_with_gloo():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    res = [out[r] for r in range(world)]
    assert res[0][1] == res[1][0] and res[0][0] == 0 and res[1][1] == 16
    total = 10 * 256 + 6 * 64
    for a, b, tmax, rate in res:
        assert tmax == 1.5
        assert abs(rate - total / 1.5) < 1e-9
