"""Multi-rank host logic on CPU: slab partition, per-slab detector rows, the
max-over-ranks timing reduction, and two gloo ranks that each reconstruct
their z-slab (FP64 oracle) from only their band of detector rows."""
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


def _scan(N=20, P=24):
    """One small seeded scan (the same on every rank)."""
    import phantom
    R = 4.0 * N
    return R, phantom.project(phantom.make_phantom(950, N, 5), R, N, N, P)


def _rank_main(rank, world, port, out):
    """Rank `rank` reconstructs its z-slab with the FP64 oracle from the
    detector rows of its band only (the rest of its projections stays zero);
    the slabs go to every rank, and the slowest rank's time is agreed on."""
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        N, P, s, D = 20, 24, 1, 2
        R, proj = _scan(N, P)
        z0, z1 = shard.slab_partition(N, world)[rank]
        v0, v1 = shard.rows_for_slab(N, N, R, z0, z1)
        rows = np.array([k * N + v for k in range(P) for v in range(v0, v1)], dtype=np.int64)
        Q = np.zeros((P, N, N), dtype=np.float64)
        Q.reshape(-1, N)[rows] = oracle.filter_rows(proj, R, rows)
        slab = oracle.fdkod_slices(Q, R, N, s, D, list(range(z0, z1)))
        t = shard.max_over_ranks(float(10 + rank))
        gathered = [None] * world
        dist.all_gather_object(gathered, (z0, z1, v1 - v0, slab))
        out[rank] = (t, gathered)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reconstruct_their_slabs_from_their_row_bands(oracle_mod):
    """Sec. 2.2: a slab of slices reads only the detector rows the b formula
    allows, so ranks that hold only those rows reconstruct their slabs exactly
    as the whole-volume oracle does (bit for bit), with no exchange."""
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()   # no fork of this multi-threaded process
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    N, P, s, D = 20, 24, 1, 2
    R, proj = _scan(N, P)
    rows = np.arange(P * N, dtype=np.int64)
    Qw = oracle_mod.filter_rows(proj, R, rows).reshape(P, N, N)
    whole = oracle_mod.fdkod(Qw, R, N, s, D)
    for rank in range(world):
        t, gathered = out[rank]
        assert t == 10 + world - 1          # slowest rank's time
        assert sorted(z for a, b, _, _ in gathered for z in range(a, b)) == list(range(N))
        for z0, z1, nrows, slab in gathered:
            assert nrows < N                # each rank held only part of the detector
            assert np.array_equal(slab, whole[z0:z1])
