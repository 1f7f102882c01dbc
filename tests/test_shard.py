"""Multi-rank host logic on CPU: slab partition, per-slab detector rows, and
the max-over-ranks timing reduction, with world_size-2 gloo process groups."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1708_07515_gb300 import shard


@pytest.mark.parametrize("N,world", [(512, 1), (512, 2), (33, 4), (3, 8), (0, 2)])
def test_slab_partition_is_a_disjoint_complete_cover(N, world):
    parts = shard.slab_partition(N, world)
    assert len(parts) == world
    covered = [z for a, b in parts for z in range(a, b)]
    assert covered == list(range(N))
    sizes = [b - a for a, b in parts]
    assert max(sizes) - min(sizes) <= 1


def test_rows_for_slab_contain_every_touched_row():
    """Brute force over the slab's voxels and a fine set of views: every row
    the bilinear sample reads (floor(v) and floor(v)+1) lies in the range."""
    N, Nv = 24, 26
    R = 1.6 * N
    beta = np.linspace(0, 2 * np.pi, 97)
    x = np.arange(N) - (N - 1) / 2
    X, Y = np.meshgrid(x, x)
    for z0, z1 in shard.slab_partition(N, 5):
        v0, v1 = shard.rows_for_slab(N, Nv, R, z0, z1)
        for zi in range(z0, z1):
            z = zi - (N - 1) / 2
            for b in beta:
                U = (R + X * math.cos(b) + Y * math.sin(b)) / R
                v = z / U + (Nv - 1) / 2
                lo, hi = np.floor(v), np.floor(v) + 1
                inside = (lo >= 0) & (hi <= Nv - 1)
                assert np.all(lo[inside] >= v0) and np.all(hi[inside] < v1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        N = 64
        z0, z1 = shard.slab_partition(N, world)[rank]
        # each rank "reconstructs" its slab: here a host stand-in, no exchange
        mine = np.arange(z0, z1)
        t = shard.max_over_ranks(float(10 + rank))
        import torch
        gathered = [None] * world
        dist.all_gather_object(gathered, mine.tolist())
        out[rank] = (t, gathered)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_cover_the_volume_and_agree_on_time():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()   # no fork of this multi-threaded process
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        t, gathered = out[rank]
        assert t == 10 + world - 1          # slowest rank's time
        assert sorted(z for part in gathered for z in part) == list(range(64))
