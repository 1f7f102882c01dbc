"""Learned angular low-pass for the decomposition (a linear FIR).

Sec. 2.1 leaves the low-pass filter open and says its choice sets the
quality.  FDK-OD is linear in the taps h[|i|] (|i| < H D): decimating with
taps h and backprojecting gives sum_i h_i B_i, where B_i is the
reconstruction obtained with the unit tap at |i|.  So the taps that bring
FDK-OD closest to full FDK (D = 1) on training scans solve a small
least-squares problem,

    minimise  sum_scans || sum_i h_i B_i - f_FDK ||^2   subject to   c . h = 1,

c = (1, 2, 2, ...) (unit gain at zero frequency, so a constant stays
constant).  Every B_i and f_FDK comes from the library's kernels (a plan with
caller taps, and the same plan with D = 1); only the H D x H D normal
equations are solved on the host.

    python -m paper_1708_07515_gb300.learn --N 512 --P 720 --s 3 --D 4

prints the taps and their held-out error next to the triangle's and the
windowed sinc's.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def constraint(n: int) -> np.ndarray:
    """c with c . h = h_0 + 2 sum_{i>0} h_i, the two-sided sum of the taps."""
    c = np.full(n, 2.0)
    c[0] = 1.0
    return c


def solve_taps(G: np.ndarray, b: np.ndarray) -> np.ndarray:
    """argmin 1/2 h^T G h - b^T h subject to c . h = 1 (KKT system)."""
    n = G.shape[0]
    c = constraint(n)
    K = np.zeros((n + 1, n + 1))
    K[:n, :n] = G
    K[:n, n] = c
    K[n, :n] = c
    rhs = np.concatenate([b, [1.0]])
    return np.linalg.solve(K, rhs)[:n]


def _slices(vol, zs):
    import torch
    return vol[torch.as_tensor(zs, device=vol.device)].double().cpu().numpy().reshape(-1)


def normal_equations(plan_taps, plan_fdk, Q, n: int, zs):
    """Gram matrix G_ij = B_i . B_j and b_i = B_i . f_FDK over slices zs of one
    scan (Q filtered, on the device)."""
    f = _slices(plan_fdk.backproject(Q), zs)
    B = np.empty((n, f.size))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        plan_taps.set_taps(e)
        B[i] = _slices(plan_taps.backproject(Q), zs)
    return B @ B.T, B @ f, B, f


def learn(R: float, N: int, P: int, s: int, D: int, H: int, train_projs, zs) -> np.ndarray:
    """Taps of half-width H D fitted on the given projections (torch CUDA
    tensors [P][N][N], unfiltered)."""
    from .fdkod import Plan
    n = H * D
    G = np.zeros((n, n))
    b = np.zeros(n)
    with Plan(R, N, N, N, P, s, D) as pt, Plan(R, N, N, N, P, s, 1) as pf:
        for proj in train_projs:
            Q = pt.filter(proj)
            g, bb, _, _ = normal_equations(pt, pf, Q, n, zs)
            G += g
            b += bb
    return solve_taps(G, b)


def held_out_errors(R: float, N: int, P: int, s: int, D: int, taps: dict, projs, zs) -> dict:
    """rel-RMSE of FDK-OD against full FDK on the given scans, per taps."""
    from .fdkod import Plan
    out = {}
    with Plan(R, N, N, N, P, s, 1) as pf:
        refs = []
        for proj in projs:
            refs.append(_slices(pf.backproject(pf.filter(proj)), zs))
        for name, h in taps.items():
            with Plan(R, N, N, N, P, s, D, taps=h) as p:
                num = den = 0.0
                for proj, f in zip(projs, refs):
                    g = _slices(p.backproject(p.filter(proj)), zs)
                    num += float(np.sum((g - f) ** 2))
                    den += float(np.sum(f ** 2))
                out[name] = (num / den) ** 0.5
    return out


def main(argv=None):
    import torch

    import phantom
    from .fdkod import fdkod_sinc_taps

    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--N", type=int, default=512)
    ap.add_argument("--P", type=int, default=720)
    ap.add_argument("--s", type=int, default=3)
    ap.add_argument("--D", type=int, default=4)
    ap.add_argument("--H", type=int, default=2, choices=[1, 2])
    ap.add_argument("--train", type=int, default=4, help="training scans (seeds 8000..)")
    ap.add_argument("--test", type=int, default=2, help="held-out scans (seeds 9000..)")
    ap.add_argument("--ellipsoids", type=int, default=40)
    ap.add_argument("--slices", type=int, default=16)
    args = ap.parse_args(argv)
    N, P, s, D, H = args.N, args.P, args.s, args.D, args.H
    R = 4.0 * N
    zs = np.linspace(N // 8, N - 1 - N // 8, args.slices).round().astype(int)

    def scans(seed0, k):
        return [phantom.project_gpu(phantom.make_phantom(seed0 + i, N, args.ellipsoids), R, N, N, P)
                for i in range(k)]

    torch.cuda.set_device(0)
    h = learn(R, N, P, s, D, H, scans(8000, args.train), zs)
    tri = (D - np.arange(D)) / float(D * D)
    errs = held_out_errors(R, N, P, s, D, {"triangle": tri, "sinc": fdkod_sinc_taps(D, 2), "learned": h},
                           scans(9000, args.test), zs)
    print(json.dumps({"N": N, "P": P, "s": s, "D": D, "H": H, "train_scans": args.train,
                      "held_out_scans": args.test, "taps": [float(x) for x in h],
                      "rel_rmse_vs_fdk": errs}))


if __name__ == "__main__":
    main()
