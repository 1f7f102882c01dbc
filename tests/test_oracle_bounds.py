"""Pins of the oracle's per-square crop bounds (Eq. 1 at the vertices, Sec. 2.1).

The brute force here projects every voxel centre of a square by intersecting
the source ray with the detector plane (vector algebra, not Eq. 1), so a
wrong sign, a transposed vertex or a dropped offset in the oracle fails.
Eq. 1 is linear-fractional in (x, y), hence monotone along any segment, so
its extremes over a square of voxel centres sit at the corner voxels: the
vertex bounds must equal the brute-force extremes, not merely contain them.
"""
import numpy as np
import pytest


def _project_u(R, Nu, P, x, y):
    """Column u of points (x, y, 0) for all views: shape [P][...]."""
    beta = 2 * np.pi * np.arange(P) / P
    S = -R * np.stack([np.cos(beta), np.sin(beta)], axis=1)        # source [P][2]
    n = np.stack([np.cos(beta), np.sin(beta)], axis=1)              # detector normal
    eu = np.stack([-np.sin(beta), np.cos(beta)], axis=1)            # detector axis
    pts = np.stack([np.ravel(x), np.ravel(y)], axis=1)              # [M][2]
    d = pts[None, :, :] - S[:, None, :]                             # [P][M][2]
    lam = -(S[:, None, :] * n[:, None, :]).sum(-1) / (d * n[:, None, :]).sum(-1)
    hit = S[:, None, :] + lam[..., None] * d
    a = (hit * eu[:, None, :]).sum(-1)
    return a + (Nu - 1) / 2


def _squares(N, s):
    m = 2 ** s
    sq = (np.arange(N) * m) // N
    return [np.nonzero(sq == q)[0] for q in range(m)]


CASES = [(8, 1, 4.0), (13, 1, 4.0), (13, 2, 1.3), (16, 2, 4.0), (33, 3, 4.0), (33, 2, 1.3), (17, 0, 2.0)]


@pytest.mark.parametrize("N,s,Rf", CASES)
def test_vertex_bounds_equal_brute_force(oracle_mod, N, s, Rf):
    P, Nu = 36, N + 3
    R = Rf * N
    b = oracle_mod.bounds(R, N, Nu, P, s)
    groups = _squares(N, s)
    m = 2 ** s
    ties = 0
    for qy in range(m):
        for qx in range(m):
            q = qy * m + qx
            xs = groups[qx] - (N - 1) / 2
            ys = groups[qy] - (N - 1) / 2
            X, Y = np.meshgrid(xs, ys)
            u = _project_u(R, Nu, P, X, Y)                   # [P][voxels]
            fl = np.floor(u)
            near = np.abs(u - np.round(u)) < 1e-9
            for k in range(P):
                lo, hi = b["lo"][q, k], b["hi"][q, k]
                # every column a voxel's linear interpolation touches lies in [lo, hi]
                assert fl[k].min() >= lo - near[k].any() and fl[k].max() + 1 <= hi + near[k].any()
                if near[k].any():
                    ties += 1
                    continue
                assert lo == fl[k].min() and hi == fl[k].max() + 1
            # phi is the projection of the square centre
            xc, yc = 0.5 * (xs[0] + xs[-1]), 0.5 * (ys[0] + ys[-1])
            pc = _project_u(R, Nu, P, np.array([xc]), np.array([yc]))[:, 0]
            np.testing.assert_allclose(b["phi"][q], pc, rtol=0, atol=1e-9)
            # the shifted grid t = u - phi - w0 keeps every voxel in [1, T-2)
            t = u - pc[:, None] - b["w0"][q]
            assert t.min() >= 1 - 1e-9 and t.max() < b["T"][q] - 2 + 1e-9
            assert t.min() < 2 + 1e-9 and t.max() > b["T"][q] - 4 - 1e-9   # and is tight
            # the crop start is the floor of the first sample position
            np.testing.assert_array_equal(b["crop"][q], np.floor(b["phi"][q] + b["w0"][q]).astype(np.int32))
    # exact integers (ties) occur only at symmetric angles; they are few
    assert ties <= max(4, P * m * m // 10)


def test_bounds_are_deterministic(oracle_mod):
    """Sec. 2.1: the formulas carry no detector row, so one bound per
    (square, angle) serves every slice; repeated calls agree bit for bit."""
    a = oracle_mod.bounds(100.0, 25, 25, 20, 2)
    b = oracle_mod.bounds(100.0, 25, 25, 20, 2)
    for key in a:
        assert np.array_equal(a[key], b[key])


def test_square_count_and_ragged_sides(oracle_mod):
    N, s = 2000, 5
    b = oracle_mod.bounds(4.0 * N, N, N, 8, s)
    assert b["lo"].shape == (4 ** s, 8)
    sides = {len(g) for g in _squares(N, s)}
    assert sides == {62, 63}


def test_rejects_bad_arguments(oracle_mod):
    with pytest.raises(RuntimeError):
        oracle_mod.bounds(100.0, 4, 4, 8, 3)     # 2^s > N
    with pytest.raises(RuntimeError):
        oracle_mod.bounds(-1.0, 16, 16, 8, 1)


@pytest.mark.parametrize("N,s,Rf,P", [(33, 2, 1.3, 36), (256, 3, 4.0, 90), (200, 2, 1.6, 60)])
def test_float32_positions_stay_inside_the_margins(oracle_mod, N, s, Rf, P):
    """The one-column margins of w0 and T are there for a backprojection
    that addresses the shifted rows in FP32: with Eq. 1, the magnification
    and the subtraction of phi and w0 all evaluated in float32, every voxel
    of every square still reads columns floor(t) >= 0 and floor(t) + 1 <=
    T - 1 of its shifted row."""
    Nu = N + 5
    R = Rf * N
    b = oracle_mod.bounds(R, N, Nu, P, s)
    f = np.float32
    beta = 2 * np.pi * np.arange(P) / P
    cb, sb = np.cos(beta).astype(f)[:, None], np.sin(beta).astype(f)[:, None]
    groups = _squares(N, s)
    m = 2 ** s
    worst_lo, worst_hi = np.inf, np.inf
    for qy in range(m):
        for qx in range(m):
            q = qy * m + qx
            X, Y = np.meshgrid(groups[qx] - (N - 1) / 2, groups[qy] - (N - 1) / 2)
            x, y = X.ravel().astype(f)[None], Y.ravel().astype(f)[None]
            u = f(R) * (y * cb - x * sb) / (f(R) + x * cb + y * sb) + f((Nu - 1) / 2)
            t = u - b["phi"][q].astype(f)[:, None] - f(b["w0"][q])
            assert t.dtype == f
            c0 = np.floor(t)
            assert c0.min() >= 0 and c0.max() + 1 <= b["T"][q] - 1
            worst_lo = min(worst_lo, float(t.min()))
            worst_hi = min(worst_hi, float(b["T"][q] - 1 - (c0.max() + 1)))
    # the margins are not wasted: some square comes within two columns of each end
    assert worst_lo < 2.0 and worst_hi <= 2
