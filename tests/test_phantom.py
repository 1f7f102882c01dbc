"""Pins of the seeded input generator (closed-form ellipsoid projector).

The projector is checked against geometry written independently here: the
sphere chord 2 sqrt(r^2 - d^2) with d the point-to-line distance, and a fine
numerical quadrature of the ellipsoid indicator along the ray.
"""
import numpy as np

import phantom


def _ray(R, Nu, Nv, P, k, u, v):
    beta = 2 * np.pi * k / P
    S = -R * np.array([np.cos(beta), np.sin(beta), 0.0])
    a, b = u - (Nu - 1) / 2, v - (Nv - 1) / 2
    T = a * np.array([-np.sin(beta), np.cos(beta), 0.0]) + b * np.array([0.0, 0.0, 1.0])
    return S, T


def test_sphere_chord_closed_form():
    rng = np.random.default_rng(1)
    R, Nu, Nv, P = 60.0, 31, 23, 12
    c = np.array([2.5, -3.0, 1.5])
    r, rho = 9.0, 0.7
    e = phantom.ellipsoid(c, [r, r, r], phantom.random_rotation(rng), rho)
    p = phantom.project(e[None], R, Nu, Nv, P, dtype=np.float64)
    for k in range(P):
        for v in range(0, Nv, 3):
            for u in range(Nu):
                S, T = _ray(R, Nu, Nv, P, k, u, v)
                d = T - S
                dist = np.linalg.norm(np.cross(c - S, d)) / np.linalg.norm(d)
                want = rho * 2 * np.sqrt(max(r * r - dist * dist, 0.0))
                assert abs(p[k, v, u] - want) < 1e-9 * max(1.0, want)


def test_ellipsoid_matches_quadrature():
    rng = np.random.default_rng(2)
    R, Nu, Nv, P = 50.0, 21, 17, 8
    rot = phantom.random_rotation(rng)
    c = np.array([1.0, 2.0, -1.5])
    ax = np.array([7.0, 4.0, 5.5])
    e = phantom.ellipsoid(c, ax, rot, 1.0)
    p = phantom.project(e[None], R, Nu, Nv, P, dtype=np.float64)
    Minv = rot @ np.diag(1.0 / ax ** 2) @ rot.T
    n = 200000
    lam = (np.arange(n) + 0.5) / n
    checked = 0
    for k in range(P):
        for v in (3, 8, 12):
            for u in range(0, Nu, 2):
                S, T = _ray(R, Nu, Nv, P, k, u, v)
                d = T - S
                # the ray segment from S to 2T - S passes the whole object
                pts = S[None, :] + (2.0 * lam)[:, None] * d[None, :] - c[None, :]
                inside = np.einsum("ni,ij,nj->n", pts, Minv, pts) <= 1.0
                want = inside.mean() * 2.0 * np.linalg.norm(d)
                assert abs(p[k, v, u] - want) < 2e-3 * max(1.0, want) + 4 * 2 * np.linalg.norm(d) / n
                checked += want > 0
    assert checked > 20


def test_rotation_by_quarter_turn_is_angle_shift():
    """Rotating the object by +90 deg about z equals shifting views by P/4."""
    N, P = 24, 16
    ell = phantom.make_phantom(11, N, 5)
    rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    rot = ell.copy()
    for e in rot:
        e[0:3] = rz @ e[0:3]
        e[6:15] = (rz @ e[6:15].reshape(3, 3)).reshape(9)
    p0 = phantom.project(ell, 4.0 * N, N, N, P, dtype=np.float64)
    p1 = phantom.project(rot, 4.0 * N, N, N, P, dtype=np.float64)
    np.testing.assert_allclose(p1, np.roll(p0, P // 4, axis=0), rtol=0, atol=1e-9)


def test_phantom_recipe_is_seeded():
    a = phantom.make_phantom(5, 64, 10)
    b = phantom.make_phantom(5, 64, 10)
    assert np.array_equal(a, b)
    assert np.all(np.linalg.norm(a[:, 0:3], axis=1) <= 0.7 * 32 + 1e-12)
    assert np.all((a[:, 3:6] >= 0.05 * 64) & (a[:, 3:6] <= 0.3 * 64))
    assert np.all((a[:, 15] >= 0.1) & (a[:, 15] <= 1.0))
    for e in a:
        q = e[6:15].reshape(3, 3)
        np.testing.assert_allclose(q @ q.T, np.eye(3), atol=1e-12)


def test_row_band_equals_the_rows_of_the_whole_detector():
    """The band projector evaluates the same rays as the whole-detector one."""
    ell = phantom.make_phantom(91, 24, 5)
    R = 80.0
    full = phantom.project(ell, R, 30, 26, 7)
    band = phantom.project(ell, R, 30, 26, 7, rows=(9, 17))
    assert band.shape == (7, 8, 30)
    assert np.array_equal(band, full[:, 9:17])
    assert phantom.project(ell, R, 30, 26, 7, k0=2, k1=5, rows=(0, 26)).shape == (3, 26, 30)
