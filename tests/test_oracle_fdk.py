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
  * linearity in the data;
  * the central slice is the 2D fan-beam FBP of the mid-plane's rays
    (closed-form ellipse chords as the scan; its own pre-weight and ramp,
    the kernel integrated numerically from the ramp spectrum; the 2D
    backprojection from vector ray geometry and the fan weight (R / L)^2,
    not from Eq. 1).
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


# ---------------------------------------------------------------------------
# Central slice = 2D fan-beam FBP.  In the mid-plane (z = 0, detector row
# b = 0) every ray of the cone lies in the plane, so FDK reduces to the
# filtered backprojection of a 2D fan-beam scan on a flat detector.  The
# input is a 2D scan of ellipses, their chords in closed form; the 2D
# backprojection below is written from the fan geometry with vectors (ray /
# detector-line intersection, the point's depth along the central ray), not
# from Eq. 1.

def _ellipse_chords(ell, S, Dp):
    """Line integrals of ellipses (cx, cy, A, B, alpha, rho) along the rays
    from points S to points Dp (arrays [..., 2])."""
    d = Dp - S
    d = d / np.linalg.norm(d, axis=-1, keepdims=True)
    n = np.stack([-d[..., 1], d[..., 0]], axis=-1)             # unit normal of the ray
    out = np.zeros(S.shape[:-1])
    for cx, cy, A, B, al, rho in ell:
        t = ((S - np.array([cx, cy])) * n).sum(-1)               # signed distance of the ray
        e1, e2 = np.array([np.cos(al), np.sin(al)]), np.array([-np.sin(al), np.cos(al)])
        a2 = A * A * (n @ e1) ** 2 + B * B * (n @ e2) ** 2      # squared support of the ellipse along n
        out += rho * 2.0 * A * B * np.sqrt(np.maximum(a2 - t * t, 0.0)) / a2
    return out


def _fan_scan(ell, R, Nu, P):
    """[P][Nu] fan-beam scan: source -R(cos b, sin b), flat detector through
    the origin along (-sin b, cos b), pitch 1, columns centred."""
    beta = 2 * np.pi * np.arange(P) / P
    a = np.arange(Nu) - (Nu - 1) / 2
    S = -R * np.stack([np.cos(beta), np.sin(beta)], -1)[:, None, :] * np.ones((1, Nu, 1))
    Dp = a[None, :, None] * np.stack([-np.sin(beta), np.cos(beta)], -1)[:, None, :]
    return _ellipse_chords(ell, S, Dp)


def _fan_filter(scan, R):
    """Fan-beam pre-weight and ramp filter of scan [P][Nu]: each sample times
    the cosine of its ray's fan angle, R / sqrt(R^2 + a^2), then a linear
    convolution along the row with the band-limited ramp of unit sample
    spacing, h(n) = (1 / 2 pi) int_{-pi}^{pi} |w| / (2 pi) e^{i w n} dw,
    whose samples are integrated numerically here."""
    from scipy.integrate import quad
    P, Nu = scan.shape
    a = np.arange(Nu) - (Nu - 1) / 2
    g = scan * (R / np.sqrt(R * R + a * a))[None]
    n = np.arange(-(Nu - 1), Nu)
    h = np.array([quad(lambda w: w, 0.0, np.pi, weight="cos", wvar=float(k))[0] if k else np.pi ** 2 / 2
                  for k in n]) / (2 * np.pi ** 2)
    return np.stack([np.convolve(row, h)[Nu - 1:2 * Nu - 1] for row in g])


def _fan_backprojection(Q, R, N):
    """2D FBP backprojection of filtered rows Q [P][Nu]: for each pixel and
    view, the detector column where the source ray through the pixel meets
    the detector line, the depth L of the pixel along the central ray, and
    the fan weight (R / L)^2; linear interpolation (zero beyond the ends);
    full-orbit redundancy 1/2 times the angular step 2 pi / P."""
    P, Nu = Q.shape
    beta = 2 * np.pi * np.arange(P) / P
    c = np.arange(N) - (N - 1) / 2
    X, Y = np.meshgrid(c, c, indexing="xy")
    pts = np.stack([X.ravel(), Y.ravel()], -1)
    cols = np.arange(-1, Nu + 1, dtype=np.float64)
    f = np.zeros(len(pts))
    for k in range(P):
        u_axis = np.array([-np.sin(beta[k]), np.cos(beta[k])])
        central = np.array([np.cos(beta[k]), np.sin(beta[k])])   # source -> origin
        S = -R * central
        d = pts - S
        L = d @ central                                           # depth along the central ray
        hit = S + d * (R / L)[:, None]                            # on the line x . central = 0
        col = hit @ u_axis + (Nu - 1) / 2
        row = np.concatenate([[0.0], Q[k], [0.0]])
        f += np.interp(col, cols, row, left=0.0, right=0.0) * (R / L) ** 2
    return (0.5 * 2 * np.pi / P) * f.reshape(N, N)


def _ellipse_density(ell, N):
    c = np.arange(N) - (N - 1) / 2
    X, Y = np.meshgrid(c, c, indexing="xy")
    f = np.zeros((N, N))
    edge = np.full((N, N), np.inf)                                # distance-like margin to any boundary
    for cx, cy, A, B, al, rho in ell:
        u = (X - cx) * np.cos(al) + (Y - cy) * np.sin(al)
        v = -(X - cx) * np.sin(al) + (Y - cy) * np.cos(al)
        r = np.sqrt((u / A) ** 2 + (v / B) ** 2)
        f += rho * (r <= 1.0)
        edge = np.minimum(edge, np.abs(r - 1.0) * min(A, B))
    return f, edge


@pytest.mark.parametrize("Rf", [1.5, 4.0])
def test_central_slice_is_fan_beam_fbp(oracle_mod, Rf):
    N, Nu, P = 41, 67, 120
    R = Rf * N
    ell = [(0.0, 0.0, 15.0, 11.0, 0.3, 1.0), (5.0, -3.0, 4.0, 6.5, -0.7, 0.5), (-6.0, 5.0, 3.5, 2.5, 1.1, -0.4)]
    scan = _fan_scan(ell, R, Nu, P).astype(np.float32)             # the oracle reads float32 scans
    Q = oracle_mod.filter(scan[:, None, :], R)                    # one detector row, b = 0
    got = oracle_mod.fdk_slices(Q, R, N, [(N - 1) // 2])[0]       # z = 0 (N odd)
    want = _fan_backprojection(_fan_filter(scan.astype(np.float64), R), R, N)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-12
    # and it is a reconstruction: pixels at least 3 voxels from every boundary
    # come back at their density, up to the discretisation error of a
    # 41-voxel grid with sharp edges (mean ~1.5 %, a few pixels ~10 %)
    dens, edge = _ellipse_density(ell, N)
    inside = edge >= 3.0
    assert inside.sum() > 500
    err = np.abs(got - dens)[inside]
    assert err.mean() <= 0.03 and np.percentile(err, 99) <= 0.15, (err.mean(), np.percentile(err, 99))
