"""Pins of the oracle's FDK-OD (Sec. 2.1 shift/decimation, Sec. 2.2 decomposition).

Independent facts used:
  * the decomposition alone changes nothing (Sec. 2.2): D = 1 with any s is
    plain FDK, bit for bit (same samples, same summation order), and every
    column read stays inside the square's crop window;
  * with s = 0 and an odd detector width the square centre projects onto a
    pixel for every view, the shift is exact, and FDK-OD reduces to plain
    FDK on the angularly low-passed views beta_{jD} (the low-pass written
    out here in numpy);
  * rotation by P/4 views rotates the volume when (P/4) mod D = 0;
  * a homogeneous centred ball still reconstructs to its density;
  * the decimation has unit DC gain and keeps a linear ramp linear;
  * the error against plain FDK grows with D (Sec. 2.2: skipping decimation
    stages improves quality).
"""
import numpy as np
import pytest

import phantom


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_D1_is_plain_fdk_bit_for_bit(oracle_mod, s):
    N, P = 16, 24
    R = 4.0 * N
    Q = np.random.default_rng(20 + s).standard_normal((P, N, N))
    assert np.array_equal(oracle_mod.fdkod(Q, R, N, s, 1), oracle_mod.fdk(Q, R, N))


def test_D1_ragged_squares_is_plain_fdk(oracle_mod):
    N, P = 13, 20
    R = 1.3 * N
    Q = np.random.default_rng(31).standard_normal((P, N + 2, N + 4))
    assert np.array_equal(oracle_mod.fdkod(Q, R, N, 2, 1), oracle_mod.fdk(Q, R, N))


@pytest.mark.parametrize("D", [2, 3, 4])
def test_s0_reduces_to_fdk_on_lowpassed_views(oracle_mod, D):
    N, P = 15, 24
    Nu, Nv = 17, 15     # odd: the isocentre projects onto a pixel centre
    R = 3.0 * N
    Q = np.random.default_rng(40 + D).standard_normal((P, Nv, Nu))
    F = np.zeros((P // D, Nv, Nu))
    for j in range(P // D):
        for i in range(-(D - 1), D):
            F[j] += (D - abs(i)) / D ** 2 * Q[(j * D + i) % P]
    got = oracle_mod.fdkod(Q, R, N, 0, D)
    want = oracle_mod.fdk(F, R, N)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("s,D", [(1, 2), (2, 4), (2, 8)])
def test_quarter_turn_equivariance(oracle_mod, s, D):
    N, P = 16, 32
    R = 4.0 * N
    Q = np.random.default_rng(50 + D).standard_normal((P, N, N))
    v0 = oracle_mod.fdkod(Q, R, N, s, D)
    v1 = oracle_mod.fdkod(np.roll(Q, P // 4, axis=0), R, N, s, D)
    want = np.empty_like(v0)
    for iy in range(N):
        for ix in range(N):
            want[:, iy, ix] = v0[:, N - 1 - ix, iy]
    np.testing.assert_allclose(v1, want, rtol=0, atol=1e-11 * np.abs(v0).max())


def test_centred_ball_keeps_its_density(oracle_mod):
    N, P = 32, 96
    R = 4.0 * N
    c, r = (0.0, 0.0, 0.0), 10.0
    e = phantom.ellipsoid(c, [r, r, r], np.eye(3), 1.0)
    Q = oracle_mod.filter(phantom.project(e[None], R, N, N, P), R)
    zi = [N // 2]
    vol = oracle_mod.fdkod_slices(Q, R, N, 2, 4, zi)[0]
    x = np.arange(N) - (N - 1) / 2
    X, Y = np.meshgrid(x, x)
    z = zi[0] - (N - 1) / 2
    d = np.sqrt(X ** 2 + Y ** 2 + z ** 2)
    assert np.abs(vol[d < r - 2] - 1).max() < 0.02


def test_decimation_dc_gain_and_ramp(oracle_mod):
    N, P, s, D = 16, 24, 1, 4
    Nu, Nv = 40, 16      # wide detector: all sample positions stay inside
    R = 4.0 * N
    const = np.broadcast_to(np.arange(Nv, dtype=np.float64)[None, :, None] + 2.0, (P, Nv, Nu)).copy()
    b = oracle_mod.bounds(R, N, Nu, P, s)
    for q in range(4):
        S = oracle_mod.shift_decimate(const, R, N, s, D, q)
        np.testing.assert_allclose(S, np.broadcast_to(const[0, None, :, :1], S.shape), rtol=0, atol=1e-13)
    ramp = np.broadcast_to(np.arange(Nu, dtype=np.float64)[None, None, :], (P, Nv, Nu)).copy()
    for q in range(4):
        S = oracle_mod.shift_decimate(ramp, R, N, s, D, q)
        # the shifted row samples u = phi + w0 + t, so each decimated row is
        # t + w0 + (a weighted mean of phi over the filter support)
        np.testing.assert_allclose(np.diff(S, axis=-1), 1.0, atol=1e-12)
        off = S[:, :, 0] - b["w0"][q]
        for j in range(P // D):
            sup = [(j * D + i) % P for i in range(-(D - 1), D)]
            assert b["phi"][q, sup].min() - 1e-12 <= off[j].min() <= off[j].max() <= b["phi"][q, sup].max() + 1e-12


def test_error_grows_with_decimation_factor(oracle_mod):
    w = phantom.Workload("t", 32, 48, 2, 1, 6, 0.0, 77)
    p = phantom.make_projections(w)
    Q = oracle_mod.filter(p, w.R)
    zs = [8, 16, 24]
    ref = oracle_mod.fdk_slices(Q, w.R, w.N, zs)
    errs = []
    for D in (1, 2, 4, 8):
        v = oracle_mod.fdkod_slices(Q, w.R, w.N, 2, D, zs)
        errs.append(np.linalg.norm(v - ref) / np.linalg.norm(ref))
    assert errs[0] == 0.0
    assert errs[1] < errs[2] < errs[3]
    assert errs[1] < 0.12


def test_error_falls_with_smaller_squares(oracle_mod):
    """Centring on a smaller square narrows its sinogram band, so at a fixed
    decimation factor the error against FDK falls as s grows (Sec. 2.2)."""
    w = phantom.Workload("t", 65, 96, 2, 1, 6, 0.0, 77)
    Q = oracle_mod.filter(phantom.make_projections(w), w.R)
    zs = [16, 32, 48]
    ref = oracle_mod.fdk_slices(Q, w.R, w.N, zs)
    errs = [np.linalg.norm(oracle_mod.fdkod_slices(Q, w.R, w.N, s, 4, zs) - ref) / np.linalg.norm(ref)
            for s in (1, 2, 3)]
    assert errs[0] > errs[1] > errs[2]


def test_slices_match_full_volume(oracle_mod):
    N, P = 16, 24
    R = 4.0 * N
    Q = np.random.default_rng(60).standard_normal((P, N, N))
    full = oracle_mod.fdkod(Q, R, N, 2, 3)
    zs = [15, 0, 7]
    assert np.array_equal(oracle_mod.fdkod_slices(Q, R, N, 2, 3, zs), full[zs])


def test_rejects_decimation_not_dividing_views(oracle_mod):
    with pytest.raises(RuntimeError):
        oracle_mod.fdkod(np.zeros((10, 8, 8)), 32.0, 8, 1, 3)
