"""Parity at the benchmark configurations' own shapes (Sec. 2.2: 4^s squares;
Sec. 3: the paper's N range), on identical inputs for the GPU and the FP64
oracle.

* The precision form's shape (s = 4 at 1024^3 gives 64-voxel squares, D = 8,
  16-bit windows) at N = 256, P = 144, s = 2, D = 8 (64-voxel squares), in
  bfloat16 and float16, whole volume.
* The precision form itself: 1024^3 from 720 views, s = 4, D = 8, bfloat16
  Q, on two seeded slices.  Only the detector rows those slices read are
  generated (a row band per slice, zero elsewhere on both sides), so the
  oracle stays bounded.
* The batched form's largest instance: N = 384, P = 538 = 2 x 269, D = 2,
  s = 3, float32, on three seeded slices.

Bars: rel-RMSE <= 1e-5 and max error <= 2e-4 max|oracle| (FP32
arithmetic; the 16-bit cases read the same rounded Q on both sides)."""
import numpy as np
import pytest

import phantom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_RMSE = 1e-5
MAX_REL = 2e-4
_TORCH16 = {"bf16": "bfloat16", "f16": "float16"}


@pytest.fixture(scope="module")
def fd():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1708_07515_gb300 as fd
    fd.load()
    return fd


def _cmp(got, want, what):
    err = got.astype(np.float64) - want
    rel = np.linalg.norm(err) / np.linalg.norm(want)
    mx = np.abs(err).max() / np.abs(want).max()
    assert rel <= REL_RMSE and mx <= MAX_REL, f"{what}: rel-RMSE {rel:.3e}, max-rel {mx:.3e}"


def _round(Q, qtype):
    """(device tensor in the storage type, the same values as float32 on the host)."""
    if qtype == "f32":
        t = torch.from_numpy(np.ascontiguousarray(Q, dtype=np.float32))
        return t.cuda(), t.numpy()
    t = torch.from_numpy(np.ascontiguousarray(Q, dtype=np.float32)).to(getattr(torch, _TORCH16[qtype]))
    return t.cuda(), t.float().numpy()


@pytest.mark.parametrize("qtype", ["bf16", "f16"])
def test_precision_form_shape_64_voxel_squares(fd, oracle_mod, qtype):
    N, P, s, D = 256, 144, 2, 8
    R = 4.0 * N
    ell = phantom.make_phantom(3000 + 7, N, 20)
    Q = oracle_mod.filter_fft(phantom.project(ell, R, N, N, P), R)
    Qd, Qr = _round(Q, qtype)
    with fd.Plan(R, N, N, N, P, s, D, qtype=qtype) as plan:
        assert plan.info["n_squares"] == 16 and N // 4 == 64
        got = plan.backproject(Qd).cpu().numpy()
        assert plan.device_status() == 0
    _cmp(got, oracle_mod.fdkod(Qr, R, N, s, D), f"FDK-OD {qtype} 256^3 s=2 D=8")


def _banded_scan(oracle_mod, N, P, n_ell, seed, zs, noise=0.0):
    """Filtered projections that hold, for each slice in zs, the detector
    rows it reads (zero elsewhere): float64 [P][N][N]."""
    R = 4.0 * N
    ell = phantom.make_phantom(seed, N, n_ell)
    Q = np.zeros((P, N, N), dtype=np.float32)
    for z in zs:
        v0, n = oracle_mod.slice_rows(R, N, N, [int(z)])
        v1 = v0 + n
        band = phantom.project(ell, R, N, N, P, rows=(v0, v1))
        if noise:
            phantom.add_noise(band, noise, seed + int(z))
        Q[:, v0:v1] = oracle_mod.filter_fft(band, R, v0=v0, Nv_det=N).astype(np.float32)
    return R, Q


def test_precision_form_1024_bf16_sampled_slices(fd, oracle_mod):
    N, P, s, D = 1024, 720, 4, 8
    zs = np.sort(np.random.default_rng(3000).choice(N, size=2, replace=False))
    R, Q = _banded_scan(oracle_mod, N, P, 80, 3000, zs)
    Qd, Qr = _round(Q, "bf16")
    del Q
    with fd.Plan(R, N, N, N, P, s, D, qtype="bf16") as plan:
        vol = plan.backproject(Qd)
        got = vol[torch.from_numpy(zs).cuda()].cpu().numpy()
        assert plan.device_status() == 0
        del vol
    _cmp(got, oracle_mod.fdkod_slices(Qr, R, N, s, D, zs), "FDK-OD bf16 1024^3 s=4 D=8")


def test_batched_form_largest_instance_sampled_slices(fd, oracle_mod):
    N, P, s, D = 384, 538, 3, 2
    zs = np.sort(np.random.default_rng(4384).choice(N, size=3, replace=False))
    R, Q = _banded_scan(oracle_mod, N, P, 20, 4384, zs)
    Qd, Qr = _round(Q, "f32")
    with fd.Plan(R, N, N, N, P, s, D) as plan:
        got = plan.backproject(Qd)[torch.from_numpy(zs).cuda()].cpu().numpy()
        plain = plan.backproject_plain(Qd)[torch.from_numpy(zs).cuda()].cpu().numpy()
        assert plan.device_status() == 0
    _cmp(got, oracle_mod.fdkod_slices(Qr, R, N, s, D, zs), "FDK-OD 384^3 P=538 D=2")
    _cmp(plain, oracle_mod.fdk_slices(Qr, R, N, zs), "plain FDK 384^3 P=538")
