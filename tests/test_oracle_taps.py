"""Pins for the angular low-pass of the decomposition (Sec. 2.1 leaves the
kernel open: the triangle is the default reading, a Hann-windowed sinc the
plan option).  The taps are checked against closed forms of their frequency
responses, and the oracle's circular filtering against the response of an
LTI filter to pure tones."""
import numpy as np
import pytest

import phantom


def _response(h, w):
    """H(w) = h0 + 2 sum_{i>0} h_i cos(i w) of symmetric taps h[|i|]."""
    i = np.arange(1, len(h))
    return h[0] + 2.0 * np.sum(h[1:, None] * np.cos(np.outer(i, np.atleast_1d(w))), axis=0)


@pytest.mark.parametrize("D", [1, 2, 3, 4, 8, 16])
def test_taps_have_unit_gain_at_zero_frequency(oracle_mod, D):
    for h in (oracle_mod.triangle_taps(D), oracle_mod.sinc_taps(D, 1), oracle_mod.sinc_taps(D, 2),
              oracle_mod.sinc_taps(D, 3)):
        assert abs(h[0] + 2 * h[1:].sum() - 1.0) < 1e-14


def test_sinc_taps_at_unit_decimation_are_the_identity(oracle_mod):
    # sinc vanishes at every non-zero integer
    for H in (1, 2, 3):
        h = oracle_mod.sinc_taps(1, H)
        assert h[0] == 1.0 and np.all(np.abs(h[1:]) < 1e-16)


@pytest.mark.parametrize("D", [2, 4, 8])
def test_triangle_response_is_the_fejer_kernel(oracle_mod, D):
    # the Bartlett window's transform: (sin(D w / 2) / (D sin(w / 2)))^2
    w = np.linspace(0.01, np.pi, 400)
    want = (np.sin(D * w / 2) / (D * np.sin(w / 2))) ** 2
    np.testing.assert_allclose(_response(oracle_mod.triangle_taps(D), w), want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("D", [2, 4, 8, 16])
def test_sinc_taps_cut_off_at_the_decimated_nyquist(oracle_mod, D):
    h, t = oracle_mod.sinc_taps(D), oracle_mod.triangle_taps(D)
    # half gain at the cutoff pi / D, flatter passband than the triangle
    assert abs(_response(h, np.pi / D)[0] - 0.5) < 0.01
    wp = np.linspace(0, 0.25 * np.pi / D, 50)
    assert _response(h, wp).min() > _response(t, wp).min()
    assert _response(h, wp).min() > 0.97


@pytest.mark.parametrize("taps", ["sinc2", "sinc1"])
def test_decimation_of_pure_tones_is_the_filter_response(oracle_mod, taps):
    """Views carrying cos(2 pi m k / P) (constant along the detector) come out
    of the circular low-pass as H(2 pi m / P) cos(2 pi m j D / P)."""
    N, P, s, D = 16, 48, 1, 4
    Nu, Nv = 40, 8      # wide detector: every shifted sample stays inside
    R = 4.0 * N
    h = oracle_mod.sinc_taps(D, 2 if taps == "sinc2" else 1)
    for m in (1, 3, 7, 11):
        w = 2 * np.pi * m / P
        Q = np.broadcast_to(np.cos(w * np.arange(P))[:, None, None], (P, Nv, Nu)).copy()
        for q in (0, 3):
            S = oracle_mod.shift_decimate(Q, R, N, s, D, q, taps=h)
            want = _response(h, w)[0] * np.cos(w * D * np.arange(P // D))
            np.testing.assert_allclose(S, np.broadcast_to(want[:, None, None], S.shape), rtol=0, atol=1e-12)


def test_explicit_triangle_taps_equal_the_default(oracle_mod):
    N, P, s, D = 24, 36, 2, 3
    R = 4.0 * N
    Q = np.random.default_rng(61).standard_normal((P, N, N))
    t = oracle_mod.triangle_taps(D)
    assert np.array_equal(oracle_mod.shift_decimate(Q, R, N, s, D, 5, taps=t), oracle_mod.shift_decimate(Q, R, N, s, D, 5))
    zs = [3, 12]
    assert np.array_equal(oracle_mod.fdkod_slices(Q, R, N, s, D, zs, taps=t), oracle_mod.fdkod_slices(Q, R, N, s, D, zs))


def test_windowed_sinc_is_closer_to_fdk_than_the_triangle(oracle_mod):
    """Less aliasing from the decimation: at the same D the windowed sinc
    reconstruction is nearer full FDK (Sec. 2.1: the low-pass filter sets the
    quality)."""
    w = phantom.Workload("t", 32, 48, 2, 4, 8, 0.0, 91)
    Q = oracle_mod.filter(phantom.make_projections(w), w.R)
    zs = [8, 16, 24]
    ref = oracle_mod.fdk_slices(Q, w.R, w.N, zs)
    err = lambda v: np.linalg.norm(v - ref) / np.linalg.norm(ref)
    e_tri = err(oracle_mod.fdkod_slices(Q, w.R, w.N, 2, 4, zs))
    e_sinc = err(oracle_mod.fdkod_slices(Q, w.R, w.N, 2, 4, zs, taps=oracle_mod.sinc_taps(4)))
    assert e_sinc < 0.97 * e_tri
