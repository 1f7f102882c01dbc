"""Pins of the oracle's plain FDK (filter + backprojection, Sec. 1 and 2.1).

Independent facts used:
  * a homogeneous ball reconstructs to its density inside and ~0 outside
    (FDK is exact in the mid-plane and nearly so for small cone angles);
    an off-centre ball pins the sign and origin of the column coordinate,
    the U^-2 weight, the pi/P scale and the row coordinate z/U; a short
    source distance (R = 1.5 N, fan half-angle ~18 deg) makes a wrong
    cosine weight or magnification visible;
  * rotating the data by P/4 views (the projector's own quarter-turn
    symmetry, pinned in test_phantom.py) rotates the volume by 90 degrees;
  * linearity in the data.
"""
import numpy as np
import pytest

import phantom


def _ball_data(oracle_mod, N, P, R, c, r, rho=1.0):
    e = phantom.ellipsoid(c, [r, r, r], np.eye(3), rho)
    p = phantom.project(e[None], R, N, N, P)
    return oracle_mod.filter(p, R)


def _dist(N, z_index, c):
    x = np.arange(N) - (N - 1) / 2
    X, Y = np.meshgrid(x, x, indexing="xy")  # [y][x]
    z = z_index - (N - 1) / 2
    return np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (z - c[2]) ** 2)


@pytest.mark.parametrize("Rf,c,r,zi", [
    (4.0, (0.0, 0.0, 0.0), 10.0, 16),
    (4.0, (6.0, -3.0, 0.0), 5.0, 16),
    (1.5, (6.0, -3.0, 0.0), 5.0, 16),
    (1.5, (-5.0, 7.0, 4.0), 5.0, 20),
    (1.5, (7.0, 5.0, -4.0), 5.0, 12),
])
def test_ball_reconstructs_to_density(oracle_mod, Rf, c, r, zi):
    N, P = 33, 128
    R = Rf * N
    rho = 0.8
    Q = _ball_data(oracle_mod, N, P, R, c, r, rho)
    vol = oracle_mod.fdk_slices(Q, R, N, [zi])[0]
    d = _dist(N, zi, c)
    rr = _dist(N, (N - 1) / 2, (0.0, 0.0, 0.0))
    # outside the ball but inside the field of view (edge streaks of a
    # 128-view scan of a small ball reach a few percent there)
    inside, outside = d < r - 2, (d > r + 3) & (rr < (N - 1) / 2 - 2)
    assert inside.sum() > 5
    assert np.abs(vol[inside] / rho - 1).max() < 0.015
    assert abs(vol[inside].mean() / rho - 1) < 0.006
    assert np.abs(vol[outside]).max() < 0.1 * rho
    assert np.sqrt(np.mean(vol[outside] ** 2)) < 0.035 * rho


def test_quarter_turn_equivariance(oracle_mod):
    N, P = 20, 32
    R = 4.0 * N
    rng = np.random.default_rng(7)
    Q = rng.standard_normal((P, N, N))
    v0 = oracle_mod.fdk(Q, R, N)
    v1 = oracle_mod.fdk(np.roll(Q, P // 4, axis=0), R, N)
    # (x, y) -> (-y, x): new[y'][x'] = old at x = y', y = -x'
    want = np.empty_like(v0)
    for iy in range(N):
        for ix in range(N):
            want[:, iy, ix] = v0[:, N - 1 - ix, iy]
    np.testing.assert_allclose(v1, want, rtol=0, atol=1e-12 * np.abs(v0).max())


def test_linearity(oracle_mod):
    N, P = 12, 16
    R = 4.0 * N
    rng = np.random.default_rng(8)
    Q1, Q2 = rng.standard_normal((2, P, N, N))
    a, b = 0.7, -1.9
    lhs = oracle_mod.fdk(a * Q1 + b * Q2, R, N)
    rhs = a * oracle_mod.fdk(Q1, R, N) + b * oracle_mod.fdk(Q2, R, N)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12 * np.abs(rhs).max())


def test_float32_and_float64_inputs_agree(oracle_mod):
    N, P = 10, 12
    R = 4.0 * N
    Q = np.random.default_rng(9).standard_normal((P, N, N)).astype(np.float32)
    assert np.array_equal(oracle_mod.fdk(Q, R, N), oracle_mod.fdk(Q.astype(np.float64), R, N))


def test_slices_equal_full_volume(oracle_mod):
    N, P = 10, 12
    R = 4.0 * N
    Q = np.random.default_rng(10).standard_normal((P, N, N))
    full = oracle_mod.fdk(Q, R, N)
    zs = [7, 0, 9, 3]
    assert np.array_equal(oracle_mod.fdk_slices(Q, R, N, zs), full[zs])


def test_off_plane_ball_lands_at_its_centre(oracle_mod):
    """A ball far off the mid-plane and off the axis (cone half-angle ~18
    degrees) is reconstructed where it is: its centroid pins the row
    coordinate v = z/U + (Nv-1)/2 (Sec. 2.2, b formula)."""
    N, P = 33, 128
    R = 1.5 * N
    c, r = (8.0, -2.0, 9.0), 4.0
    Q = _ball_data(oracle_mod, N, P, R, c, r)
    vol = oracle_mod.fdk(Q, R, N)
    x = np.arange(N) - (N - 1) / 2
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    d = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    w = np.clip(vol, 0, None) * (d < r + 3)
    got = [(w * A).sum() / w.sum() for A in (X, Y, Z)]
    np.testing.assert_allclose(got, c, atol=0.1)
    assert abs(vol[d < r - 1.5].mean() - 1) < 0.03
