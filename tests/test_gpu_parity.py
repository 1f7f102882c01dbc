"""GPU parity: the CUDA library (called through its C ABI) against the FP64
oracle, element by element on the same seeded inputs.

Bars:
  * crop bounds (integers and the FP64 shift centres): bit-exact;
  * filter: per row, max |Q_gpu - Q_oracle| <= 2 log2(L) 2^-24 ||q_pair||_2
    (FFT round-off grows with log2 L times the input norm, the ramp's gain
    is at most 1/2, and two rows share one complex transform, so each row's
    round-off scales with the norm of its pair);
  * backprojections (FP32 path): rel-RMSE = ||g - o|| / ||o|| <= 1e-5 over
    the compared voxels, and max |g - o| <= 2e-4 max |o|.
Inputs: seeded random-ellipsoid phantoms (phantom module), their exact
projections, filtered by the oracle in FP64 and rounded to float32 so both
sides read identical Q values.
"""
import glob
import os

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


def _q_from_phantom(oracle_mod, N, P, n_ell, seed, noise=0.0, R=None, Nu=None, Nv=None, fft=False):
    R = 4.0 * N if R is None else R
    Nu = N if Nu is None else Nu
    Nv = N if Nv is None else Nv
    ell = phantom.make_phantom(seed, N, n_ell)
    p = phantom.project(ell, R, Nu, Nv, P)
    if noise:
        phantom.add_noise(p, noise, seed)
    Q = oracle_mod.filter_fft(p, R) if fft else oracle_mod.filter(p, R)
    return p, Q.astype(np.float32), R


def _cmp(got, want, what):
    err = got.astype(np.float64) - want
    rel = np.linalg.norm(err) / np.linalg.norm(want)
    mx = np.abs(err).max() / np.abs(want).max()
    assert rel <= REL_RMSE and mx <= MAX_REL, f"{what}: rel-RMSE {rel:.3e}, max-rel {mx:.3e}"
    return rel, mx


BOUND_CASES = [
    # R, N, Nu, P, s
    (512.0, 128, 128, 128, 2),
    (2048.0, 512, 512, 720, 3),
    (4096.0, 1024, 1024, 720, 4),
    (8000.0, 2000, 2000, 720, 5),
    (1.3 * 33, 33, 37, 36, 3),
    (200.0, 50, 51, 90, 2),
    (64.0, 16, 16, 8, 0),
]


@pytest.mark.parametrize("R,N,Nu,P,s", BOUND_CASES)
def test_bounds_bit_exact(fd, oracle_mod, R, N, Nu, P, s):
    plan = fd.Plan(R, N, Nu, N, P, s, 1)
    got = plan.bounds()
    want = oracle_mod.bounds(R, N, Nu, P, s)
    for key in ("lo", "hi", "crop", "w0", "T"):
        assert np.array_equal(got[key], want[key]), key
    assert np.array_equal(got["phi"].view(np.int64), want["phi"].view(np.int64))
    plan.close()


GOLDEN = sorted(glob.glob(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bounds_*.txt")))


@pytest.mark.parametrize("path", GOLDEN, ids=os.path.basename)
def test_bounds_equal_the_stored_fixtures(fd, path):
    """The library's bounds against the stored oracle values of
    tests/golden (no oracle call at run time)."""
    from test_golden import _read
    g = _read(path)
    R, N, Nu, P, s = g["geometry"]
    plan = fd.Plan(R, N, Nu, N, P, s, 1)
    got = plan.bounds()
    for key in ("lo", "hi", "crop", "w0", "T"):
        assert np.array_equal(got[key], g[key]), key
    assert np.array_equal(got["phi"].view(np.int64), g["phi"].view(np.int64))
    plan.close()


@pytest.mark.parametrize("N,Nu,Nv,P", [(32, 32, 32, 16), (50, 53, 47, 12), (128, 128, 128, 8), (512, 512, 512, 4),
                                       (1000, 1000, 3, 2)])
def test_filter_parity(fd, oracle_mod, N, Nu, Nv, P):
    R = 4.0 * N
    ell = phantom.make_phantom(100 + N, N, 8)
    p = phantom.project(ell, R, Nu, Nv, P)
    plan = fd.Plan(R, N, Nu, Nv, P, 0, 1)
    Qg = plan.filter(torch.from_numpy(p).cuda()).cpu().numpy().astype(np.float64)
    Qo = oracle_mod.filter(p, R)
    a = np.arange(Nu) - (Nu - 1) / 2
    b = np.arange(Nv) - (Nv - 1) / 2
    q = p.astype(np.float64) * (R / np.sqrt(R * R + a[None, :] ** 2 + b[:, None] ** 2))[None]
    L = plan.info["fft_length"]
    rn = np.linalg.norm(q, axis=-1).reshape(-1)          # flat row order k * Nv + v
    pair = np.sqrt(np.add.reduceat(rn ** 2, np.arange(0, rn.size, 2)))
    tol = 2 * np.log2(L) * 2.0 ** -24 * np.repeat(pair, 2)[:rn.size]
    err = np.abs(Qg - Qo).max(axis=-1).reshape(-1)
    assert np.all(err <= tol), (err / np.maximum(tol, 1e-300)).max()
    plan.close()


PLAIN_CASES = [
    # N, P, Nu, Nv, R factor
    (33, 36, 33, 33, 4.0),     # ragged tiles
    (50, 60, 53, 47, 1.5),     # short source distance, non-square detector
    (64, 64, 64, 64, 4.0),
    (128, 128, 128, 128, 4.0),  # the 128^3, P = 128 workload
]


@pytest.mark.parametrize("N,P,Nu,Nv,Rf", PLAIN_CASES)
def test_plain_fdk_parity(fd, oracle_mod, N, P, Nu, Nv, Rf):
    _, Q, R = _q_from_phantom(oracle_mod, N, P, 10, 200 + N, R=Rf * N, Nu=Nu, Nv=Nv)
    plan = fd.Plan(R, N, Nu, Nv, P, 0, 1)
    vol = plan.backproject_plain(torch.from_numpy(Q).cuda()).cpu().numpy()
    want = oracle_mod.fdk(Q, R, N)
    _cmp(vol, want, "plain FDK")
    assert plan.device_status() == 0
    plan.close()


FDKOD_CASES = [
    # N, P, s, D, Nu, Nv, R factor
    (128, 128, 2, 2, 128, 128, 4.0),   # the 128^3, P = 128, s = 2, D = 2 workload
    (64, 96, 3, 4, 64, 64, 4.0),
    (50, 60, 2, 3, 53, 47, 1.5),       # ragged squares (12/13), odd D
    (33, 36, 1, 6, 33, 33, 4.0),
    (64, 64, 2, 1, 64, 64, 4.0),       # D = 1: crop only
    (40, 48, 0, 2, 41, 41, 4.0),       # s = 0
    (64, 32, 2, 32, 64, 64, 4.0),      # one decimated view
    (96, 64, 1, 4, 100, 90, 4.0),      # decomposed rows of 65..128 columns (32 lanes per row)
    (96, 48, 0, 2, 96, 96, 4.0),       # rows past 128 columns (8 columns per lane)
    (125, 144, 1, 16, 125, 125, 4.0),  # ragged 62/63-voxel squares at D = 16 (the 2000^3 square size)
    (125, 144, 1, 24, 125, 125, 4.0),  # and at D = 24
]


@pytest.mark.parametrize("N,P,s,D,Nu,Nv,Rf", FDKOD_CASES)
def test_fdkod_parity(fd, oracle_mod, N, P, s, D, Nu, Nv, Rf):
    _, Q, R = _q_from_phantom(oracle_mod, N, P, 10, 300 + N + D, R=Rf * N, Nu=Nu, Nv=Nv)
    plan = fd.Plan(R, N, Nu, Nv, P, s, D)
    vol = plan.backproject(torch.from_numpy(Q).cuda()).cpu().numpy()
    want = oracle_mod.fdkod(Q, R, N, s, D)
    _cmp(vol, want, f"FDK-OD s={s} D={D}")
    assert plan.device_status() == 0
    plan.close()


@pytest.mark.parametrize("N,P,s,D", [(64, 96, 3, 4), (50, 60, 2, 3), (32, 32, 1, 2), (96, 48, 0, 2), (96, 64, 1, 4)])
def test_decomposed_data_parity(fd, oracle_mod, N, P, s, D):
    _, Q, R = _q_from_phantom(oracle_mod, N, P, 6, 400 + N)
    plan = fd.Plan(R, N, N, N, P, s, D)
    S = plan.decompose(torch.from_numpy(Q).cuda()).cpu().numpy()
    T = plan.bounds()["T"]
    for q in sorted({0, 4 ** s // 2, 4 ** s - 1}):
        want = oracle_mod.shift_decimate(Q, R, N, s, D, q)
        got = S[q, :, :, :T[q]].astype(np.float64)
        assert np.abs(got - want).max() <= 1e-6 * np.abs(Q).max(), q
        assert np.all(S[q, :, :, T[q]:] == 0)
    plan.close()


def test_repeated_calls_are_deterministic(fd, oracle_mod):
    _, Q, R = _q_from_phantom(oracle_mod, 64, 96, 6, 500)
    plan = fd.Plan(R, 64, 64, 64, 96, 3, 4)
    Qd = torch.from_numpy(Q).cuda()
    a = plan.backproject(Qd).cpu()
    b = plan.backproject(Qd).cpu()
    assert torch.equal(a, b)
    plan.close()


def test_full_size_512_sampled_slices(fd, oracle_mod):
    """512^3 from 720 views of 512^2, s = 3, D = 4, 40 ellipsoids + 1 % noise:
    full volumes on the GPU, the oracle on seeded slices."""
    w = phantom.WORKLOADS["fdkod_512"]
    _, Q, R = _q_from_phantom(oracle_mod, w.N, w.P, w.n_ell, w.seed, noise=w.noise, fft=True)
    rng = np.random.default_rng(w.seed)
    zs = np.sort(rng.choice(w.N, size=4, replace=False))
    plan = fd.Plan(R, w.N, w.N, w.N, w.P, w.s, w.D)
    Qd = torch.from_numpy(Q).cuda()
    od = plan.backproject(Qd)[torch.from_numpy(zs).cuda()].cpu().numpy()
    pl = plan.backproject_plain(Qd)[torch.from_numpy(zs).cuda()].cpu().numpy()
    assert plan.device_status() == 0
    _cmp(od, oracle_mod.fdkod_slices(Q, R, w.N, w.s, w.D, zs), "FDK-OD 512")
    _cmp(pl, oracle_mod.fdk_slices(Q, R, w.N, zs), "plain FDK 512")
    plan.close()


# ---- precision forms: Q stored as bfloat16 / float16 (FP32 arithmetic) ----

_TORCH16 = {"bf16": "bfloat16", "f16": "float16"}


def _round16(Q, qtype):
    t = torch.from_numpy(Q.astype(np.float32)).to(getattr(torch, _TORCH16[qtype]))
    return t, t.float().numpy()


@pytest.mark.parametrize("qtype", ["bf16", "f16"])
@pytest.mark.parametrize("N,P,s,D,Nu,Nv", [(64, 96, 3, 4, 64, 64), (50, 60, 2, 3, 53, 47), (128, 128, 2, 2, 128, 128),
                                            (96, 64, 1, 4, 96, 96), (96, 48, 0, 2, 96, 96)])
def test_precision_forms_parity_on_identical_inputs(fd, oracle_mod, qtype, N, P, s, D, Nu, Nv):
    """Both sides read the same 16-bit-rounded Q; the arithmetic is FP32 on
    the GPU and FP64 in the oracle, so the FP32 bar applies."""
    _, Q, R = _q_from_phantom(oracle_mod, N, P, 10, 600 + N + D, Nu=Nu, Nv=Nv)
    Q16, Qr = _round16(Q, qtype)
    plan = fd.Plan(R, N, Nu, Nv, P, s, D, qtype=qtype)
    Qd = Q16.cuda()
    _cmp(plan.backproject(Qd).cpu().numpy(), oracle_mod.fdkod(Qr, R, N, s, D), f"FDK-OD {qtype}")
    _cmp(plan.backproject_plain(Qd).cpu().numpy(), oracle_mod.fdk(Qr, R, N), f"plain FDK {qtype}")
    assert plan.device_status() == 0
    plan.close()


@pytest.mark.parametrize("qtype", ["bf16", "f16"])
def test_filter_writes_16bit_within_rounding(fd, oracle_mod, qtype):
    N, P = 64, 16
    R = 4.0 * N
    p = phantom.project(phantom.make_phantom(700, N, 8), R, N, N, P)
    plan = fd.Plan(R, N, N, N, P, 0, 1, qtype=qtype)
    Qg = plan.filter(torch.from_numpy(p).cuda()).float().cpu().numpy().astype(np.float64)
    Qo = oracle_mod.filter(p, R)
    # round-to-nearest storage: half an ulp, 2^-9 (bf16) or 2^-12 (f16)
    # relative, plus the f16 subnormal spacing and the FFT round-off
    rel = 2.0 ** -8 if qtype == "bf16" else 2.0 ** -11
    fft = 2 * np.log2(plan.info["fft_length"]) * 2.0 ** -24 * 2 * np.abs(Qo).max() * np.sqrt(N)
    assert np.all(np.abs(Qg - Qo) <= rel * np.abs(Qo) + 2.0 ** -24 + fft)
    plan.close()


@pytest.mark.parametrize("qtype,bound", [("bf16", 5e-3), ("f16", 1e-3)])
def test_precision_form_error_against_fp64(fd, oracle_mod, qtype, bound):
    """The storage rounding's own cost: 16-bit Q against the FP64 oracle on
    unrounded Q (the bench states the measured value per workload)."""
    N, P, s, D = 64, 96, 3, 4
    _, Q, R = _q_from_phantom(oracle_mod, N, P, 10, 800)
    Q16, _ = _round16(Q, qtype)
    plan = fd.Plan(R, N, N, N, P, s, D, qtype=qtype)
    got = plan.backproject(Q16.cuda()).cpu().numpy().astype(np.float64)
    want = oracle_mod.fdkod(Q, R, N, s, D)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel < bound, rel
    plan.close()
