"""Pins of the oracle's filter stage (cosine weight + Ram-Lak convolution).

What mathematics fixes, independent of the oracle's code:
  * the discrete Ram-Lak kernel with unit spacing is the band-limited ramp,
    so a long cosine row of frequency f (cycles/sample) comes out scaled by
    |f| away from the row ends;
  * its taps sum to zero over the whole line (the ramp vanishes at f = 0);
    for a finite row of ones the output is the two truncated tails,
    ~ (1/pi^2) (1/(2 L1) + 1/(2 L2)) with L1, L2 the distances to the ends;
  * the weight R / sqrt(R^2 + a^2 + b^2) is the cosine of the ray angle, so
    a row equal to 1 / weight behaves like a row of ones.
"""
import numpy as np
import pytest


def _inv_weight(R, Nu, Nv):
    a = np.arange(Nu) - (Nu - 1) / 2
    b = np.arange(Nv) - (Nv - 1) / 2
    return np.sqrt(R * R + a[None, :] ** 2 + b[:, None] ** 2) / R  # [Nv][Nu]


@pytest.mark.parametrize("f0", [0.031, 0.125, 0.29, 0.43])
def test_ramp_response_of_cosine(oracle_mod, f0):
    Nu, Nv, R = 4001, 5, 700.0  # short R: the cosine weight varies by ~2 % across b
    m = np.arange(Nu)
    row = np.cos(2 * np.pi * f0 * m + 0.3)
    proj = (row[None, :] * _inv_weight(R, Nu, Nv)).astype(np.float32)[None]
    # float32 rounding of the input adds ~1e-7 to the response
    Q = oracle_mod.filter(proj, R)[0]
    mid = slice(1000, 3001)
    want = abs(f0) * np.cos(2 * np.pi * f0 * m[mid] + 0.3)
    # the truncated kernel's tail beyond 1000 samples is bounded by
    # sum_{|n|>1000} 1/(pi^2 n^2) < 1e-4 and oscillates against the cosine
    err = np.abs(Q[:, mid] - want[None, :]).max()
    assert err < 1e-5, err


def test_dc_response_is_the_truncated_tail(oracle_mod):
    Nu, R = 1001, 1e6
    proj = np.ones((1, 1, Nu), np.float32)
    Q = oracle_mod.filter(proj, R)[0, 0]
    for u in (100, 300, 500, 700, 900):
        L1, L2 = u + 0.5, Nu - 1 - u + 0.5
        want = (1 / (2 * L1) + 1 / (2 * L2)) / np.pi ** 2
        # midpoint estimate of sum over odd n > L of 1/n^2; relative
        # residual O(1/L)
        assert abs(Q[u] - want) < 0.01 * want, (u, Q[u], want)


def test_cosine_weight_uses_both_detector_coordinates(oracle_mod):
    Nu, Nv, R = 601, 301, 150.0
    proj = _inv_weight(R, Nu, Nv).astype(np.float64)
    proj32 = proj.astype(np.float32)[None]
    Q = oracle_mod.filter(proj32, R)[0]
    ones = oracle_mod.filter(np.ones((1, 1, Nu), np.float32), 1e9)[0, 0]
    # float32 rounding of 1/weight is ~6e-8 relative, times |h| summed (<=1/2)
    np.testing.assert_allclose(Q, np.broadcast_to(ones, Q.shape), rtol=0, atol=1e-6)


def test_matches_fft_convolution_with_ramp_spectrum(oracle_mod):
    """Zero-padded FFT filtering with the ramp |f| sampled in the frequency
    domain converges to the same linear convolution as the padding grows;
    compare at 16x padding, away from aliasing."""
    rng = np.random.default_rng(3)
    Nu, Nv, P, R = 64, 3, 2, 256.0
    proj = rng.standard_normal((P, Nv, Nu)).astype(np.float32)
    Q = oracle_mod.filter(proj, R)
    q = proj.astype(np.float64) / _inv_weight(R, Nu, Nv)[None]
    # the kernel's DTFT is |f| on [-1/2, 1/2]; its samples on a fine grid of
    # length L give the circular convolution with the periodised kernel,
    # whose aliasing error is O(1/L^2)
    L = 1 << 16
    f = np.fft.fftfreq(L)
    H = np.abs(f)
    X = np.fft.fft(q, n=L, axis=-1)
    y = np.real(np.fft.ifft(X * H, axis=-1))[..., :Nu]
    assert np.abs(Q - y).max() < 1e-8


@pytest.mark.parametrize("Nu,Nv", [(17, 5), (64, 3), (100, 7)])
def test_fft_form_equals_direct_convolution(oracle_mod, Nu, Nv):
    rng = np.random.default_rng(Nu)
    proj = (10 * rng.random((3, Nv, Nu))).astype(np.float32)
    R = 3.0 * Nu
    a = oracle_mod.filter(proj, R)
    b = oracle_mod.filter_fft(proj, R)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-12 * np.abs(proj).max())


def test_fft_form_on_a_row_band_equals_the_direct_rows(oracle_mod):
    """A band of rows filtered on its own (each row with its own cosine
    weight b = v - (Nv-1)/2) equals the direct convolution of those rows of
    the whole detector."""
    rng = np.random.default_rng(31)
    P, Nv, Nu, R = 3, 40, 37, 90.0
    proj = rng.standard_normal((P, Nv, Nu)).astype(np.float32)
    v0, v1 = 11, 29
    band = oracle_mod.filter_fft(proj[:, v0:v1], R, v0=v0, Nv_det=Nv)
    np.testing.assert_allclose(band, oracle_mod.filter(proj, R)[:, v0:v1], rtol=0, atol=1e-12)
    with pytest.raises(ValueError):
        oracle_mod.filter_fft(proj[:, v0:v1], R, v0=30, Nv_det=Nv)
