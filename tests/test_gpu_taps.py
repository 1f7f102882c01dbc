"""GPU parity of the angular low-pass options (Sec. 2.1 leaves the filter
open): the windowed-sinc plan flag and caller-given taps, against the FP64
oracle with the same taps, through every decomposition path (TMA lane
shapes, 16-bit storage, slab-wise reconstruction).  Bars as in
test_gpu_parity.py."""
import numpy as np
import pytest

import phantom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_RMSE = 1e-5
MAX_REL = 2e-4


@pytest.fixture(scope="module")
def fd():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1708_07515_gb300 as fd
    fd.load()
    return fd


def _q(oracle_mod, N, P, seed, Nu=None, Nv=None, n_ell=8):
    R = 4.0 * N
    p = phantom.project(phantom.make_phantom(seed, N, n_ell), R, Nu or N, Nv or N, P)
    return oracle_mod.filter(p, R).astype(np.float32), R, p


def _cmp(got, want, what):
    err = got.astype(np.float64) - want
    rel = np.linalg.norm(err) / np.linalg.norm(want)
    mx = np.abs(err).max() / np.abs(want).max()
    assert rel <= REL_RMSE and mx <= MAX_REL, f"{what}: rel-RMSE {rel:.3e}, max-rel {mx:.3e}"


@pytest.mark.parametrize("N,P,s,D,Nu,Nv", [
    (64, 96, 3, 4, 64, 64),     # 8 lanes per row
    (50, 60, 2, 3, 53, 47),     # ragged squares, odd D, generic path for a 53-column detector
    (33, 36, 1, 6, 33, 33),     # support 2D = 12 of 36 views
    (64, 64, 2, 16, 64, 64),    # support 2D = 32: half the orbit
    (96, 64, 1, 4, 96, 96),     # 32 lanes per row
    (96, 48, 0, 2, 96, 96),     # 8 columns per lane
])
def test_sinc_taps_parity(fd, oracle_mod, N, P, s, D, Nu, Nv):
    Q, R, _ = _q(oracle_mod, N, P, 700 + N + D, Nu, Nv)
    with fd.Plan(R, N, Nu, Nv, P, s, D, taps="sinc") as plan:
        np.testing.assert_allclose(plan.taps, oracle_mod.sinc_taps(D), rtol=0, atol=1e-15)
        vol = plan.backproject(torch.from_numpy(Q).cuda()).cpu().numpy()
        assert plan.device_status() == 0
    _cmp(vol, oracle_mod.fdkod(Q, R, N, s, D, taps=oracle_mod.sinc_taps(D)), f"sinc s={s} D={D}")


@pytest.mark.parametrize("n_blocks", [1, 2])
def test_caller_taps_parity(fd, oracle_mod, n_blocks):
    N, P, s, D = 64, 96, 2, 4
    Q, R, _ = _q(oracle_mod, N, P, 710 + n_blocks)
    h = np.random.default_rng(720 + n_blocks).uniform(0.0, 1.0, n_blocks * D)
    h /= h[0] + 2 * h[1:].sum()
    with fd.Plan(R, N, N, N, P, s, D, taps=h) as plan:
        np.testing.assert_array_equal(plan.taps, h)
        Qd = torch.from_numpy(Q).cuda()
        vol = plan.backproject(Qd).cpu().numpy()
        S = plan.decompose(Qd).cpu().numpy()
        T = plan.bounds()["T"]
    _cmp(vol, oracle_mod.fdkod(Q, R, N, s, D, taps=h), f"caller taps ({n_blocks * D})")
    for q in (0, 7, 15):
        want = oracle_mod.shift_decimate(Q, R, N, s, D, q, taps=h)
        assert np.abs(S[q, :, :, :T[q]] - want).max() <= 1e-6 * np.abs(Q).max(), q


def test_triangle_taps_given_explicitly_equal_the_default(fd, oracle_mod):
    N, P, s, D = 64, 96, 3, 4
    Q, R, _ = _q(oracle_mod, N, P, 730)
    Qd = torch.from_numpy(Q).cuda()
    with fd.Plan(R, N, N, N, P, s, D) as a, fd.Plan(R, N, N, N, P, s, D, taps=oracle_mod.triangle_taps(D)) as b:
        np.testing.assert_array_equal(a.taps, oracle_mod.triangle_taps(D))
        assert torch.equal(a.backproject(Qd), b.backproject(Qd))


@pytest.mark.parametrize("qtype", ["bf16", "f16"])
def test_sinc_taps_with_16bit_storage(fd, oracle_mod, qtype):
    N, P, s, D = 64, 96, 2, 4
    Q, R, _ = _q(oracle_mod, N, P, 740)
    Qt = torch.from_numpy(Q).to(getattr(torch, {"bf16": "bfloat16", "f16": "float16"}[qtype]))
    with fd.Plan(R, N, N, N, P, s, D, qtype=qtype, taps="sinc") as plan:
        vol = plan.backproject(Qt.cuda()).cpu().numpy()
    _cmp(vol, oracle_mod.fdkod(Qt.float().numpy(), R, N, s, D, taps=oracle_mod.sinc_taps(D)), f"sinc {qtype}")


def test_sinc_taps_slab_wise(fd, oracle_mod):
    N, P, s, D = 64, 96, 3, 4
    Q, R, p = _q(oracle_mod, N, P, 750)
    with fd.Plan(R, N, N, N, P, s, D, workspace=False, taps="sinc") as plan:
        got = fd.reconstruct_slabs(plan, p, 16)
        assert plan.device_status() == 0
    want = oracle_mod.fdkod(oracle_mod.filter(p, R), R, N, s, D, taps=oracle_mod.sinc_taps(D))
    _cmp(got, want, "sinc slab-wise")


def test_taps_are_rejected_when_malformed(fd):
    with fd.Plan(256.0, 64, 64, 64, 96, 2, 4) as plan:
        for bad in (np.ones(3), np.ones(12), np.array([1.0, np.nan, 0.0, 0.0])):
            with pytest.raises(fd.FdkodError):
                fd.fdkod_set_decimation_taps(plan.handle, bad)
    with fd.Plan(256.0, 64, 64, 64, 96, 2, 1) as plan:   # D = 1: nothing to filter
        with pytest.raises(fd.FdkodError):
            fd.fdkod_set_decimation_taps(plan.handle, np.ones(1))
