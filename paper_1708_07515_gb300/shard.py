"""Host-side partitioning of one reconstruction over several GPUs.

FDK-OD needs no exchange between GPUs: voxels of different slabs are
disjoint, and a slab of slices z0..z1 reads only the detector rows the row
formula b = z R / (R + x cos b + y sin b) of Sec. 2.2 can reach, so each rank
receives only those rows of the filtered projections and writes its slab.
The functions here are pure host logic (no GPU work).
"""
from __future__ import annotations

import math


def slab_partition(N: int, world: int) -> list[tuple[int, int]]:
    """Contiguous slabs [z0, z1) of N slices for `world` ranks, sizes
    differing by at most one; ranks beyond N get empty slabs."""
    if N < 0 or world <= 0:
        raise ValueError("N >= 0 and world > 0 required")
    base, extra = divmod(N, world)
    out, z = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


def rows_for_slab(N: int, Nv: int, R: float, z0: int, z1: int) -> tuple[int, int]:
    """Detector rows [v0, v1) that slices z0..z1-1 can touch (bilinear
    interpolation included): with the in-slice radius r <= (N-1)/sqrt(2),
    U = (R + x cos b + y sin b)/R lies in [1 - r/R, 1 + r/R] and the row is
    z/U + (Nv-1)/2."""
    if z1 <= z0:
        return (0, 0)
    rmax = math.sqrt(2.0) * 0.5 * (N - 1)
    if not R > rmax:
        raise ValueError("source inside the volume")
    vc = 0.5 * (Nv - 1)
    lo, hi = math.inf, -math.inf
    for zi in (z0, z1 - 1):
        z = zi - 0.5 * (N - 1)
        for U in (1.0 - rmax / R, 1.0 + rmax / R):
            v = z / U + vc
            lo, hi = min(lo, v), max(hi, v)
    v0 = max(0, int(math.floor(lo)))
    v1 = min(Nv, int(math.floor(hi)) + 2)
    return (v0, max(v0, v1))


def max_over_ranks(value: float, group=None) -> float:
    """Largest value over the process group (the job's time is its slowest
    rank's); returns the value itself without torch.distributed."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
