"""Pins for the oracle's learned angular decimation (oracle/net.py) and the
per-square pieces it runs through (shift_rows, bp_square and its adjoint).

The net itself is pinned by an explicit-loop restatement on tiny inputs,
by positive homogeneity (no biases), by central differences of its
vector-Jacobian product, and by a closed reduction: under weights that
route +x and -x through paired channels (relu(u) - relu(-u) = u) it is a
linear FIR whose offsets are the sum of the three layers' offsets, so the
whole FDK-OD pipeline with it must equal the C oracle's FDK-OD with the
plain taps plus that FIR.  Each layer's offset is asymmetric, so a
flipped tap order, a transposed channel index or a wrong stride in any one
layer breaks the equality."""
import numpy as np
import pytest

import phantom
from oracle import net


def _rand_net(seed, scale=0.3):
    return np.random.default_rng(seed).standard_normal(net.NET_SIZE) * scale


def test_forward_matches_explicit_loops():
    rng = np.random.default_rng(1)
    for P, D, B in [(12, 3, 3), (10, 2, 2), (16, 4, 2)]:
        x = rng.standard_normal((P, B))
        w = _rand_net(P)
        np.testing.assert_allclose(net.net_forward(x, D, w), net.net_loop(x, D, w), rtol=0, atol=1e-12)


def test_positive_homogeneity_and_zero():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((24, 5))
    w = _rand_net(3)
    y = net.net_forward(x, 4, w)
    for a in (0.5, 3.0, 1e3):
        np.testing.assert_allclose(net.net_forward(a * x, 4, w), a * y, rtol=1e-12, atol=1e-12 * a)
    assert np.all(net.net_forward(np.zeros_like(x), 4, w) == 0.0)


def test_circular_shift_by_D_shifts_the_output():
    """The net is a convolution along a closed orbit: rotating the views by
    D rotates the decimated output by one."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal((30, 4))
    w = _rand_net(5)
    np.testing.assert_allclose(net.net_forward(np.roll(x, 3, axis=0), 3, w),
                               np.roll(net.net_forward(x, 3, w), 1, axis=0), rtol=0, atol=1e-12)


@pytest.mark.parametrize("D", [2, 3, 4])
def test_vjp_matches_central_differences(D):
    rng = np.random.default_rng(10 + D)
    P, B = 24, 6
    x = rng.standard_normal((P, B))
    w = _rand_net(20 + D)
    dy = rng.standard_normal((P // D, B))
    g = net.net_vjp(x, D, w, dy)
    eps = 1e-6
    for i in range(4):
        v = rng.standard_normal(net.NET_SIZE)
        lp = np.sum(dy * net.net_forward(x, D, w + eps * v))
        lm = np.sum(dy * net.net_forward(x, D, w - eps * v))
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g @ v) <= 1e-6 * max(1.0, abs(fd)), (fd, g @ v)
    # per-layer blocks: a direction inside one layer only
    for lo, hi in [(0, 80), (80, 1360), (1360, 1440)]:
        v = np.zeros(net.NET_SIZE)
        v[lo:hi] = rng.standard_normal(hi - lo)
        fd = (np.sum(dy * net.net_forward(x, D, w + eps * v)) - np.sum(dy * net.net_forward(x, D, w - eps * v))) / (
            2 * eps)
        assert abs(fd - g @ v) <= 1e-6 * max(1.0, abs(fd))


def test_linear_configuration_is_a_shifted_fir():
    rng = np.random.default_rng(30)
    P, D, B = 24, 4, 3
    x = rng.standard_normal((P, B))
    g3 = np.array([0.1, -0.2, 0.3, 0.7, -0.4])
    y = net.net_forward(x, D, net.linear_net(g3, offsets=(1, -2)))
    want = np.zeros((P // D, B))
    for j in range(P // D):
        for m in range(5):
            want[j] += g3[m] * x[(j * D + m - 2 + 1 - 2) % P]
    np.testing.assert_allclose(y, want, rtol=0, atol=1e-13)


def test_shift_rows_at_s0_is_an_integer_crop(oracle_mod):
    """s = 0: the shift centre is the detector centre for every view (an
    integer column for an odd detector), so the shifted rows are plain
    column crops of Q."""
    N, P = 13, 16
    R = 4.0 * N
    Q = np.random.default_rng(40).standard_normal((P, N, N))
    b = oracle_mod.bounds(R, N, N, P, 0)
    S = oracle_mod.shift_rows(Q, R, N, 0, 0)
    T, c = int(b["T"][0]), b["crop"][0]
    for k in range(P):
        cols = c[k] + np.arange(T)
        inside = (cols >= 0) & (cols < N)
        want = np.zeros((N, T))
        want[:, inside] = Q[k][:, cols[inside]]
        np.testing.assert_array_equal(S[k], want)


def test_shift_rows_then_circular_lowpass_is_shift_decimate(oracle_mod):
    N, P, s, D = 16, 24, 1, 4
    R = 4.0 * N
    Q = np.random.default_rng(41).standard_normal((P, N, N))
    h = oracle_mod.triangle_taps(D)
    for q in (0, 3):
        S = oracle_mod.shift_rows(Q, R, N, s, q)
        want = sum((h[abs(i)] * np.roll(S, -i, axis=0))[::D] for i in range(-(D - 1), D))
        np.testing.assert_allclose(oracle_mod.shift_decimate(Q, R, N, s, D, q), want, rtol=0, atol=1e-13)


def test_bp_square_sums_to_fdkod(oracle_mod):
    """The per-square backprojection of each square's decomposed data, summed
    over the squares, is FDK-OD (the same sums: bit for bit)."""
    N, P, s, D = 16, 24, 2, 3
    R = 4.0 * N
    Q = np.random.default_rng(42).standard_normal((P, N, N))
    zs = [0, 5, 15]
    vol = sum(oracle_mod.bp_square(oracle_mod.shift_decimate(Q, R, N, s, D, q), R, N, N, P, s, D, q, zs)
              for q in range(16))
    np.testing.assert_array_equal(vol, oracle_mod.fdkod_slices(Q, R, N, s, D, zs))


def test_bp_square_adjoint_dot_product(oracle_mod):
    """<B S, E> = <S, B^T E> for random S and E."""
    N, P, s, D = 16, 24, 1, 4
    R = 4.0 * N
    Nv = 14
    rng = np.random.default_rng(43)
    zs = [1, 8, 14]
    for q in range(4):
        T = int(oracle_mod.bounds(R, N, N, P, s)["T"][q])
        S = rng.standard_normal((P // D, Nv, T))
        E = rng.standard_normal((len(zs), N, N))
        lhs = np.sum(oracle_mod.bp_square(S, R, N, N, P, s, D, q, zs) * E)
        rhs = np.sum(S * oracle_mod.bp_square_adjoint(E, R, N, N, Nv, P, s, D, q, zs))
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_net_pipeline_with_zero_last_layer_is_plain_fdkod(oracle_mod):
    N, P, s, D = 16, 24, 1, 4
    R = 4.0 * N
    Q = phantom.project(phantom.make_phantom(44, N, 5), R, N, N, P)
    Q = oracle_mod.filter(Q, R)
    w = _rand_net(45)
    w[1360:] = 0.0
    zs = [2, 7, 13]
    np.testing.assert_allclose(oracle_mod.fdkod_net_slices(Q, R, N, s, D, w, zs),
                               oracle_mod.fdkod_slices(Q, R, N, s, D, zs), rtol=0, atol=1e-12)


@pytest.mark.parametrize("D,offsets,g3", [
    (4, (1, -2), [0.0, 0.0, 0.06, -0.1, 0.06]),   # composite offsets -1, 0, +1
    (3, (-1, 2), [0.05, 0.08, 0.05, 0.0, 0.0]),   # -1 .. +1 through other taps
    (4, (2, -1), [0.04, -0.03, 0.07, 0.0, 0.0]),  # -1 .. +1, asymmetric
])
def test_linear_net_pipeline_equals_fdkod_with_summed_taps(oracle_mod, D, offsets, g3):
    """FDK-OD with the linear net configuration = the C oracle's FDK-OD with
    taps h[|i|] = triangle + the composite FIR (when that FIR is symmetric),
    and = FDK-OD plus the backprojection of the shifted-FIR output otherwise."""
    N, P, s = 16, 24, 1
    R = 4.0 * N
    Q = oracle_mod.filter(phantom.project(phantom.make_phantom(46, N, 5), R, N, N, P), R)
    zs = [3, 8, 12]
    w = net.linear_net(g3, offsets=offsets)
    got = oracle_mod.fdkod_net_slices(Q, R, N, s, D, w, zs)
    o = offsets[0] + offsets[1]
    comp = {m - 2 + o: g for m, g in enumerate(g3) if g != 0.0}
    if all(abs(comp.get(-i, 0.0) - comp.get(i, 0.0)) < 1e-15 for i in comp):
        h = oracle_mod.triangle_taps(D).copy()
        for i, g in comp.items():
            if i >= 0:
                assert i < D
                h[i] += g
        want = oracle_mod.fdkod_slices(Q, R, N, s, D, zs, taps=h)
    else:
        want = oracle_mod.fdkod_slices(Q, R, N, s, D, zs)
        for q in range(4):
            S = oracle_mod.shift_rows(Q, R, N, s, q)
            fir = sum(g * np.roll(S, -i, axis=0) for i, g in comp.items())[::D]
            want += oracle_mod.bp_square(fir, R, N, N, P, s, D, q, zs)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-11 * np.abs(want).max())


def test_round_bf16_matches_the_format():
    """Values with 8 significant bits are fixed points; midpoints go to the
    even neighbour; the relative change is at most 2^-8."""
    exact = np.array([1.0, 1.5, 1.9921875, 3.0, 0.75, 2.0 ** -20 * 1.25, 255.0, 256.0])
    np.testing.assert_array_equal(net.round_bf16(exact), exact)
    # 1 + 2^-8 is the midpoint between 1 and 1 + 2^-7: ties to even (1)
    assert net.round_bf16(1.0 + 2.0 ** -8) == 1.0
    assert net.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2 * 2.0 ** -7     # midpoint, odd below
    assert net.round_bf16(1.0 + 2.0 ** -8 + 2.0 ** -30) == 1.0 + 2.0 ** -7
    a = np.random.default_rng(50).uniform(1e-3, 1e3, 10000)
    r = net.round_bf16(a)
    assert np.all(np.abs(r - a) <= 2.0 ** -8 * a)
    f = np.frexp(r)[0] * 256.0                          # significand as an integer
    assert np.all(f == np.round(f))


def test_act_rounding_bound_covers_bf16_storage():
    rng = np.random.default_rng(51)
    for D in (2, 4, 7):
        x = rng.standard_normal((56, 30)) * 10.0 ** rng.uniform(-2, 2)
        w = _rand_net(52 + D)
        d = np.abs(net.net_forward(x, D, w, act_round="bf16") - net.net_forward(x, D, w))
        b = net.act_rounding_bound(x, D, w)
        assert np.all(d <= b)
        assert d.max() > 0


def test_act_rounding_bound_each_layer():
    """Inputs built so that only one layer's input is off the BF16 grid: the
    bound's term for that layer alone must cover the change (x exact and a1
    exact: only a2 rounds; x off-grid with an identity-like layer 1: x and
    a1 round)."""
    rng = np.random.default_rng(53)
    P, D = 40, 4
    x = net.round_bf16(rng.standard_normal((P, 12)))          # on the BF16 grid
    W1 = np.zeros((16, 5))
    for c in range(16):
        W1[c, c % 5] = 1.0 if c % 2 == 0 else -1.0             # a1 = relu(+-x[k + m - 2]): on the grid
    W2 = rng.standard_normal((16, 16, 5)) * 0.3                 # z2 off the grid: only a2 rounds
    W3 = rng.standard_normal((16, 5)) * 0.3
    w = net.net_pack(W1, W2, W3)
    d = np.abs(net.net_forward(x, D, w, act_round="bf16") - net.net_forward(x, D, w))
    b = net.act_rounding_bound(x, D, w)
    assert d.max() > 0
    assert np.all(d <= b)
    # x off the grid, same weights: x (and so a1) round as well
    x2 = rng.standard_normal((P, 12))
    d2 = np.abs(net.net_forward(x2, D, w, act_round="bf16") - net.net_forward(x2, D, w))
    assert np.all(d2 <= net.act_rounding_bound(x2, D, w))
