"""Learned angular taps (a linear FIR fitted to full FDK): the constrained
least-squares solve on the host, and on the GPU the property the fit
guarantees -- on its training scans no taps of the same support (the
triangle and the windowed sinc among them) come closer to full FDK."""
import numpy as np
import pytest

import phantom
from paper_1708_07515_gb300 import learn


def test_constrained_solve_recovers_known_taps():
    rng = np.random.default_rng(5)
    n = 8
    B = rng.standard_normal((n, 500))
    h = rng.uniform(0, 1, n)
    h /= learn.constraint(n) @ h
    f = h @ B
    got = learn.solve_taps(B @ B.T, B @ f)
    np.testing.assert_allclose(got, h, rtol=0, atol=1e-10)


def test_constrained_solve_keeps_unit_gain():
    rng = np.random.default_rng(6)
    n = 6
    B = rng.standard_normal((n, 300))
    f = rng.standard_normal(300)          # not in the span: a true compromise
    h = learn.solve_taps(B @ B.T, B @ f)
    assert abs(learn.constraint(n) @ h - 1.0) < 1e-12
    # no other unit-gain taps fit better
    for _ in range(20):
        d = rng.standard_normal(n)
        d -= (learn.constraint(n) @ d) / (learn.constraint(n) @ learn.constraint(n)) * learn.constraint(n)
        assert np.sum(((h + 1e-3 * d) @ B - f) ** 2) >= np.sum((h @ B - f) ** 2) - 1e-9


@pytest.mark.gpu
def test_learned_taps_are_best_on_their_training_scans():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1708_07515_gb300 as fd
    N, P, s, D, H = 64, 96, 2, 4, 2
    R = 4.0 * N
    zs = [16, 32, 48]
    projs = [torch.from_numpy(phantom.project(phantom.make_phantom(8100 + i, N, 10), R, N, N, P)).cuda()
             for i in range(3)]
    h = learn.learn(R, N, P, s, D, H, projs, zs)
    tri = np.concatenate([(D - np.arange(D)) / float(D * D), np.zeros(D)])
    errs = learn.held_out_errors(R, N, P, s, D, {"triangle": tri, "sinc": fd.fdkod_sinc_taps(D, 2), "learned": h},
                                 projs, zs)
    assert errs["learned"] <= errs["triangle"] * (1 + 1e-6)
    assert errs["learned"] <= errs["sinc"] * (1 + 1e-6)
    assert abs(learn.constraint(H * D) @ h - 1.0) < 1e-9


def test_net_linear_configuration_is_the_fir():
    """learn_net.linear_config: the net (evaluated by the oracle) adds
    exactly the 13-tap FIR it was given, at every output view."""
    from oracle import net as onet

    from paper_1708_07515_gb300.learn_net import linear_config
    rng = np.random.default_rng(70)
    g = {o: float(rng.standard_normal()) for o in range(-6, 7)}
    w = linear_config(g, 3).astype(np.float64)
    for P, D in ((48, 4), (60, 3), (64, 16)):
        x = rng.standard_normal((P, 5))
        want = sum(c * np.roll(x, -o, axis=0) for o, c in g.items())[::D]
        np.testing.assert_allclose(onet.net_forward(x, D, w), want, rtol=0, atol=1e-5 * np.abs(want).max())


def test_net_trainer_host_logic():
    """learn_net's host pieces: the row-interval union, Adam's first step
    (sign of the gradient times the step size), and the zero-gain FIR
    correction recovering a planted one from its normal equations."""
    from paper_1708_07515_gb300 import learn_net
    assert learn_net.merge_rows([(5, 9), (0, 3), (8, 12), (3, 4)]) == [(0, 4), (5, 12)]
    assert learn_net.merge_rows([]) == []
    opt = learn_net.Adam(4, lr=0.01)
    w = opt.step(np.zeros(4, np.float32), np.array([1.0, -2.0, 0.5, 0.0]))
    np.testing.assert_allclose(w, [-0.01, 0.01, -0.01, 0.0], atol=1e-6)
    # a random SPD Gram matrix over 8 taps, a base filter, and a target made
    # from base + g_true with c . g_true = 0: the solve recovers g_true
    rng = np.random.default_rng(71)
    A = rng.standard_normal((40, 8))
    G = A.T @ A
    base = np.array([0.25, 0.1875, 0.125, 0.0625, 0, 0, 0, 0])
    n = 7
    g_true = rng.standard_normal(n)
    c = learn.constraint(n)
    g_true -= c * (c @ g_true) / (c @ c)
    total = base.copy()
    total[:n] += g_true
    b = G @ total                       # the normal equations' right side for that optimum
    g = learn_net.solve_correction(G, b, base, n)
    # the unconstrained optimum satisfies the constraint, so it is returned
    np.testing.assert_allclose(g, g_true, atol=1e-9)
    assert abs(c @ g) < 1e-12
    w0 = learn_net.init_weights(3)
    assert w0.shape == (1440,) and np.all(w0[1360:] == 0.0)
