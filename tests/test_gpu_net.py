"""Learned angular decimation on the GPU against the FP64 oracle
(oracle/net.py): the tensor-core inference kernel behind fdkod_decompose /
fdkod_backproject, and the training kernels (adjoint of the
backprojection, backward pass of the net).

Bars.  The kernel feeds every layer's input (x, a1, a2) to the tensor cores
as BF16, so it is compared with the oracle that rounds the same values to
BF16: what remains is FP32 arithmetic and the rare value whose FP32 and
FP64 pre-images round to neighbouring BF16 values (one BF16 step there).
Elementwise the difference must stay within the rigorous bound of one BF16
rounding of every such value (oracle.net.act_rounding_bound) plus FP32
slack, and in norm within REL_NET of the data: an isolated one-step flip
moves a few dozen outputs by ~2^-8 of their net term, so the flips among
10^5 outputs stay well below it, while a wrong tap, channel or view index
moves every output by the size of the net term.  The weights are BF16
values, so the kernel's BF16 weight storage is exact."""
import numpy as np
import pytest

import phantom
from oracle import net as onet

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_NET = 2e-4
FP32_SLACK = 1e-5


@pytest.fixture(scope="module")
def fd():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1708_07515_gb300 as fd
    fd.load()
    return fd


def _bf16_net(seed, s1=0.4, s2=0.15, s3=0.08):
    rng = np.random.default_rng(seed)
    w = np.concatenate([rng.standard_normal(80) * s1, rng.standard_normal(1280) * s2, rng.standard_normal(80) * s3])
    return onet.round_bf16(w)


def _scan(oracle_mod, seed, N, Nu, Nv, P, R, n_ell=6):
    p = phantom.project(phantom.make_phantom(seed, N, n_ell), R, Nu, Nv, P)
    return oracle_mod.filter(p, R).astype(np.float32)


def _cmp_decomposed(got, oracle_mod, Q, R, N, s, D, w, taps=None, what="", tight=True):
    """tight: the norm bar REL_NET.  With 16-bit Q the shifted samples are
    interpolations between 16-bit values and often land on a BF16 rounding
    tie, where FP32 and FP64 decide differently far more often; the norm bar
    is then the RMS of independent roundings, at most the bound's norm over
    sqrt(3)."""
    Qo = Q.astype(np.float32)
    for q in range(4 ** s):
        T = int(oracle_mod.bounds(R, N, Q.shape[2], Q.shape[0], s)["T"][q])
        want = oracle_mod.net_decomposed(Qo, R, N, s, D, q, w, taps, act_round="bf16")
        bound = onet.act_rounding_bound(oracle_mod.shift_rows(Qo, R, N, s, q), D, w)
        g = got[q, :, :, :T].astype(np.float64)
        err = np.abs(g - want)
        scale = np.abs(want).max()
        assert np.all(err <= bound + FP32_SLACK * scale), f"{what} q={q}: {(err - bound).max():.3e}"
        if tight:
            rel = np.linalg.norm(g - want) / np.linalg.norm(want)
            assert rel <= REL_NET, f"{what} q={q}: rel {rel:.3e}"
        else:
            assert np.linalg.norm(g - want) <= np.linalg.norm(bound) / np.sqrt(3.0) + \
                FP32_SLACK * np.linalg.norm(want), what
        assert np.all(got[q, :, :, T:] == 0.0)


@pytest.mark.parametrize("N,Nu,Nv,P,s,D,taps,qtype", [
    (32, 32, 32, 48, 1, 4, "triangle", "f32"),     # two column groups, ragged
    (40, 44, 36, 72, 2, 3, "triangle", "f32"),     # odd D, odd sizes
    (32, 32, 24, 64, 1, 16, "triangle", "f32"),    # 4 output views per chunk
    (32, 32, 24, 96, 1, 2, "sinc", "f32"),         # 2D-tap plain low-pass
    (24, 24, 20, 24, 1, 4, "triangle", "f32"),     # orbit shorter than one chunk
    (32, 32, 20, 120, 1, 60, "triangle", "f32"),   # largest D: one view per chunk
    (32, 32, 32, 48, 1, 4, "triangle", "bf16"),    # 16-bit Q
    (40, 44, 36, 72, 2, 3, "triangle", "f16"),
])
def test_net_decompose_matches_oracle(fd, oracle_mod, N, Nu, Nv, P, s, D, taps, qtype):
    R = 4.0 * N
    Q = _scan(oracle_mod, 900 + N + D, N, Nu, Nv, P, R)
    w = _bf16_net(901 + D)
    Qd = torch.from_numpy(Q).cuda()
    with fd.Plan(R, N, Nu, Nv, P, s, D, qtype=qtype, taps=taps) as plan:
        h = plan.taps
        plan.set_net(w)
        np.testing.assert_array_equal(plan.net, w.astype(np.float32))
        Qp = Qd.to(plan.q_torch_dtype)
        got = plan.decompose(Qp).cpu().numpy()
        assert plan.device_status() == 0
    Qref = Qp.float().cpu().numpy()   # the values the kernel read (16-bit storage rounds Q)
    _cmp_decomposed(got, oracle_mod, Qref, R, N, s, D, w, taps=h, what=f"{qtype} D={D}", tight=qtype == "f32")


def test_linear_net_configuration_equals_plain_taps(fd, oracle_mod):
    """Weights that make the net a linear FIR (paired +-x channels): the
    decomposition equals the plain one with the FIR added to the taps, up to
    the BF16 storage of a1 = relu(+-x) (bounded as above)."""
    N, P, s, D = 32, 48, 1, 4
    R = 4.0 * N
    Q = _scan(oracle_mod, 910, N, N, N, P, R)
    g3 = onet.round_bf16(np.array([0.0, 0.0, 0.0625, -0.125, 0.0625]))
    w = onet.linear_net(g3, offsets=(1, -2))
    h = oracle_mod.triangle_taps(D).copy()
    h[0] += g3[3]
    h[1] += g3[2]
    Qd = torch.from_numpy(Q).cuda()
    with fd.Plan(R, N, N, N, P, s, D) as pn, fd.Plan(R, N, N, N, P, s, D, taps=h) as pt:
        pn.set_net(w)
        a = pn.decompose(Qd).cpu().numpy().astype(np.float64)
        b = pt.decompose(Qd).cpu().numpy().astype(np.float64)
    bn = 0.0
    for q in range(4):
        bound = onet.act_rounding_bound(oracle_mod.shift_rows(Q, R, N, s, q), D, w)
        T = bound.shape[-1]
        assert np.all(np.abs(a[q, :, :, :T] - b[q, :, :, :T]) <= bound + FP32_SLACK * np.abs(b).max())
        bn += np.sum(bound ** 2)
    # here the plain side has no BF16 rounding: each output differs by a sum
    # of three independent roundings (at most 2^-8 |x| each, about uniform),
    # whose RMS is at most the bound / sqrt(3)
    assert np.linalg.norm(a - b) <= np.sqrt(bn / 3.0) + FP32_SLACK * np.linalg.norm(b)


def test_zero_last_layer_and_removal_give_the_plain_decomposition(fd, oracle_mod):
    N, P, s, D = 32, 48, 1, 4
    R = 4.0 * N
    Q = torch.from_numpy(_scan(oracle_mod, 920, N, N, N, P, R)).cuda()
    w = _bf16_net(921)
    w[1360:] = 0.0
    with fd.Plan(R, N, N, N, P, s, D) as plan:
        plain = plan.decompose(Q).clone()
        plan.set_net(w)
        zero = plan.decompose(Q).clone()
        plan.set_net(None)
        assert plan.net is None
        again = plan.decompose(Q)
    assert torch.equal(again, plain)
    # the same sums in another order: FP32 rounding only
    assert (zero - plain).norm() / plain.norm() <= 1e-6


def test_net_backprojection_matches_oracle(fd, oracle_mod):
    N, P, s, D = 32, 64, 2, 4
    R = 4.0 * N
    Q = _scan(oracle_mod, 930, N, N, N, P, R, n_ell=8)
    w = _bf16_net(931)
    zs = [0, 9, 16, 31]
    with fd.Plan(R, N, N, N, P, s, D) as plan:
        plan.set_net(w)
        vol = plan.backproject(torch.from_numpy(Q).cuda()).cpu().numpy()
        assert plan.device_status() == 0
    want = oracle_mod.fdkod_net_slices(Q, R, N, s, D, w, zs, act_round="bf16")
    got = vol[zs].astype(np.float64)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel <= REL_NET, rel
    # and the net changed the result (it is not the plain decomposition)
    plain = oracle_mod.fdkod_slices(Q, R, N, s, D, zs)
    assert np.linalg.norm(plain - want) / np.linalg.norm(want) > 50 * rel


def test_net_slab_pipeline_uses_the_net(fd, oracle_mod):
    """fdkod_reconstruct_slabs decomposes with the net as well."""
    N, P, s, D = 32, 48, 1, 4
    R = 4.0 * N
    proj = phantom.project(phantom.make_phantom(940, N, 6), R, N, N, P).astype(np.float32)
    w = _bf16_net(941)
    with fd.Plan(R, N, N, N, P, s, D, workspace=True) as plan:
        plan.set_net(w)
        Q = plan.filter(torch.from_numpy(proj).cuda())
        whole = plan.backproject(Q).cpu().numpy()
        slabs = fd.reconstruct_slabs(plan, proj, 8)
    # per-slab filtering pairs rows differently in the FFT: FP32 round-off of
    # Q, which now and then moves a net input across a BF16 rounding
    # boundary (one BF16 step of one value there, as in the oracle bars)
    assert np.linalg.norm(slabs - whole) / np.linalg.norm(whole) <= REL_NET


# ---------------------------------------------------------------- training

def test_net_adjoint_matches_oracle(fd, oracle_mod):
    N, P, s, D = 32, 48, 1, 4
    R = 4.0 * N
    rng = np.random.default_rng(950)
    with fd.Plan(R, N, N, N, P, s, D) as plan:
        info = plan.info
        T = oracle_mod.bounds(R, N, N, P, s)["T"]
        dS = torch.zeros((info["n_squares"], info["Pd"], N, info["T_stride"]), device="cuda")
        err = torch.zeros(1, device="cuda")
        zs = [3, 17, 30]
        vols = rng.standard_normal((len(zs), N, N)).astype(np.float32)
        refs = rng.standard_normal((len(zs), N, N)).astype(np.float32)
        for i, z in enumerate(zs):
            plan.net_adjoint(torch.from_numpy(vols[i]).cuda(), torch.from_numpy(refs[i]).cuda(), z, dS, err)
        torch.cuda.synchronize()
        got = dS.cpu().numpy().astype(np.float64)
    E = vols.astype(np.float64) - refs
    assert abs(err.item() - np.sum(E ** 2)) <= 1e-5 * np.sum(E ** 2)
    for q in range(4):
        want = oracle_mod.bp_square_adjoint(E, R, N, N, N, P, s, D, q, zs)
        g = got[q, :, :, :T[q]]
        assert np.linalg.norm(g - want) / np.linalg.norm(want) <= 1e-5
        assert np.all(got[q, :, :, T[q]:] == 0.0)


@pytest.mark.parametrize("D,rows", [(4, (0, 32)), (3, (5, 19))])
def test_net_backward_matches_oracle_vjp(fd, oracle_mod, D, rows):
    N, P, s = 32, 48, 1
    R = 4.0 * N
    Q = _scan(oracle_mod, 960 + D, N, N, N, P, R)
    rng = np.random.default_rng(961)
    w = (rng.standard_normal(onet.NET_SIZE) * 0.2).astype(np.float32)
    T = oracle_mod.bounds(R, N, N, P, s)["T"]
    with fd.Plan(R, N, N, N, P, s, D) as plan:
        info = plan.info
        # a coherent gradient (that of (1/2)|S'|^2 for the plain S'): the
        # weight gradients are sums of mostly like-signed terms, so the few
        # ReLU decisions that FP32 and FP64 take differently (|z| within
        # round-off of 0) change them by ~1/n; with random signs one such
        # term would already be ~1/sqrt(n) of the result
        dS = np.zeros((info["n_squares"], info["Pd"], N, info["T_stride"]), np.float32)
        for q in range(4):
            dS[q, :, :, :T[q]] = oracle_mod.shift_decimate(Q, R, N, s, D, q)
        dW = torch.zeros(onet.NET_SIZE, device="cuda")
        plan.net_backward(torch.from_numpy(Q).cuda(), torch.from_numpy(w).cuda(), torch.from_numpy(dS).cuda(),
                          rows[0], rows[1], dW)
        got = dW.cpu().numpy().astype(np.float64)
    want = np.zeros(onet.NET_SIZE)
    for q in range(4):
        x = oracle_mod.shift_rows(Q, R, N, s, q, rows[0], rows[1] - rows[0])
        want += onet.net_vjp(x, D, w.astype(np.float64), dS[q, :, rows[0]:rows[1], :T[q]].astype(np.float64))
    # FP32 sums of ~10^5 products per weight; per-layer blocks checked on their own
    for lo, hi in [(0, 80), (80, 1360), (1360, 1440)]:
        rel = np.linalg.norm(got[lo:hi] - want[lo:hi]) / np.linalg.norm(want[lo:hi])
        assert rel <= 1e-4, (lo, hi, rel)


def test_net_plans_that_cannot_take_it(fd):
    """D = 1 (no decimation) and D above 60 reject a net; non-finite weights
    and a wrong size are argument errors; a net-less plan reports none."""
    with fd.Plan(128.0, 32, 32, 32, 48, 1, 1) as p1:
        with pytest.raises(fd.FdkodError) as e:
            p1.set_net(np.zeros(onet.NET_SIZE, np.float32))
        assert e.value.status == -2
        assert p1.net is None
    with fd.Plan(128.0, 32, 32, 32, 128, 1, 64) as p64:
        with pytest.raises(fd.FdkodError) as e:
            p64.set_net(np.zeros(onet.NET_SIZE, np.float32))
        assert e.value.status == -2
    with fd.Plan(128.0, 32, 32, 32, 48, 1, 4) as p4:
        bad = np.zeros(onet.NET_SIZE, np.float32)
        bad[7] = np.nan
        for w in (bad, np.zeros(10, np.float32)):
            with pytest.raises(fd.FdkodError) as e:
                p4.set_net(w)
            assert e.value.status == -1
        assert p4.net is None


def test_net_with_taps_changed_after_setting_it(fd, oracle_mod):
    """Setting new plain taps after the net keeps the net and uses the new
    taps for the plain low-pass it adds to."""
    N, P, s, D = 32, 48, 1, 4
    R = 4.0 * N
    Q = _scan(oracle_mod, 970, N, N, N, P, R)
    w = _bf16_net(971)
    h = oracle_mod.sinc_taps(D, 2)
    with fd.Plan(R, N, N, N, P, s, D) as plan:
        plan.set_net(w)
        plan.set_taps(h)
        got = plan.decompose(torch.from_numpy(Q).cuda()).cpu().numpy()
        np.testing.assert_array_equal(plan.net, w.astype(np.float32))
    _cmp_decomposed(got, oracle_mod, Q, R, N, s, D, w, taps=h, what="taps after net")


def test_full_size_512_net_sampled_slices(fd, oracle_mod):
    """512^3 from 720 views of 512^2, s = 3, D = 4, 40 ellipsoids + 1 % noise,
    with the package's trained D = 4 weights on top of their learned linear
    taps (the bench's --taps net configuration): full volume on the GPU, the
    BF16-emulating oracle with the same taps on the two central slices (only
    the detector rows they touch are decomposed)."""
    import os
    w = phantom.WORKLOADS["fdkod_512"]
    R = 4.0 * w.N
    proj = phantom.make_projections(w)
    zs = np.array([w.N // 2 - 1, w.N // 2])   # few detector rows: a cheap oracle
    wdir = os.path.join(os.path.dirname(fd.__file__), "net_weights")
    weights = np.load(os.path.join(wdir, "D4.npy"))
    base = np.load(os.path.join(wdir, "D4_taps.npy"))
    assert base.shape == (2 * w.D,) and abs(base[0] + 2 * base[1:].sum() - 1.0) < 1e-9   # unit DC gain
    with fd.Plan(R, w.N, w.N, w.N, w.P, w.s, w.D, taps=base) as plan:
        plan.set_net(weights)
        Qd = plan.filter(torch.from_numpy(proj).cuda())
        vol = plan.backproject(Qd)[torch.from_numpy(zs).cuda()].cpu().numpy().astype(np.float64)
        assert plan.device_status() == 0
        Q = Qd.cpu().numpy()                 # the filtered data both sides read
        wq = plan.net
    want = oracle_mod.fdkod_net_slices(Q, R, w.N, w.s, w.D, wq, zs, taps=base, act_round="bf16")
    rel = np.linalg.norm(vol - want) / np.linalg.norm(want)
    assert rel <= REL_NET, rel
