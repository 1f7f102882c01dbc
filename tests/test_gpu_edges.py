"""Edge cases of the GPU path against the FP64 oracle: the smallest volumes
(one voxel, squares of one voxel), wide detectors up to the widest the
filter takes (Nu = 8192), a source just outside the volume's circumscribed cylinder and
a nearly parallel beam, one view; plans that must be rejected or that run
out of device memory; two plans working concurrently.  Bars as in
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


def _cmp(got, want, what):
    err = got.astype(np.float64) - want
    rel = np.linalg.norm(err) / np.linalg.norm(want)
    mx = np.abs(err).max() / np.abs(want).max()
    assert rel <= REL_RMSE and mx <= MAX_REL, f"{what}: rel-RMSE {rel:.3e}, max-rel {mx:.3e}"


@pytest.mark.parametrize("N,P,s,D,Nu,Nv", [
    (1, 8, 0, 2, 4, 4),      # one voxel
    (2, 8, 1, 2, 4, 4),      # squares of one voxel
    (3, 12, 1, 3, 5, 3),     # ragged squares (1 and 2 voxels), odd detector
    (5, 1, 1, 1, 8, 8),      # one view
])
def test_tiny_volumes(fd, oracle_mod, N, P, s, D, Nu, Nv):
    R = 4.0 * N + 2.0
    Q = np.random.default_rng(800 + N).standard_normal((P, Nv, Nu)).astype(np.float32)
    Qd = torch.from_numpy(Q).cuda()
    with fd.Plan(R, N, Nu, Nv, P, s, D) as plan:
        od = plan.backproject(Qd).cpu().numpy()
        pl = plan.backproject_plain(Qd).cpu().numpy()
        assert plan.device_status() == 0
    _cmp(od, oracle_mod.fdkod(Q, R, N, s, D), f"FDK-OD N={N}")
    _cmp(pl, oracle_mod.fdk(Q, R, N), f"plain FDK N={N}")


@pytest.mark.parametrize("R", [None, 1000.0 * 32])
def test_extreme_source_distances(fd, oracle_mod, R):
    """R just above the limit sqrt(2) N / 2 + 1 (magnification ~20: one
    view's window outgrows shared memory, so the unstaged kernel runs) and a
    nearly parallel beam."""
    N, P, s, D = 32, 48, 2, 4
    R = np.sqrt(2.0) * N / 2 + 1.2 if R is None else R
    p = phantom.project(phantom.make_phantom(810, N, 6), R, N, N, P)
    Q = oracle_mod.filter(p, R).astype(np.float32)
    Qd = torch.from_numpy(Q).cuda()
    with fd.Plan(R, N, N, N, P, s, D) as plan:
        od = plan.backproject(Qd).cpu().numpy()
        pl = plan.backproject_plain(Qd).cpu().numpy()
        assert plan.device_status() == 0
    _cmp(od, oracle_mod.fdkod(Q, R, N, s, D), f"FDK-OD R={R:.1f}")
    _cmp(pl, oracle_mod.fdk(Q, R, N), f"plain FDK R={R:.1f}")


@pytest.mark.parametrize("Nu,L", [(2048, 4096), (2500, 8192), (8192, 16384)])
def test_widest_detector_filter(fd, oracle_mod, Nu, L):
    """Wide detectors up to the limit: Nu = 2048 (L = 4096, 256 threads per
    row pair), 2500 (the widest the paper's experiments reach, L = 8192) and
    8192 (L = 16384, 1024 threads per row pair)."""
    N, Nv, P = 64, 6, 3
    R = 4.0 * N
    proj = np.random.default_rng(820).uniform(0.0, 1.0, (P, Nv, Nu)).astype(np.float32)
    with fd.Plan(R, N, Nu, Nv, P, 0, 1) as plan:
        assert plan.info["fft_length"] == L
        Q = plan.filter(torch.from_numpy(proj).cuda()).cpu().numpy()
    want = oracle_mod.filter(proj, R)
    # FFT round-off bar of test_gpu_parity.py: 2 log2(L) 2^-24 times the norm
    # of the cosine-weighted row pair sharing one transform
    a = np.arange(Nu) - (Nu - 1) / 2
    b = np.arange(Nv) - (Nv - 1) / 2
    q = proj.astype(np.float64) * (R / np.sqrt(R * R + a[None, :] ** 2 + b[:, None] ** 2))[None]
    rn = np.linalg.norm(q, axis=-1).reshape(-1)
    pair = np.repeat(np.sqrt(np.add.reduceat(rn ** 2, np.arange(0, rn.size, 2))), 2)[:rn.size]
    err = np.abs(Q.astype(np.float64) - want).max(axis=-1).reshape(-1)
    assert np.all(err <= 2 * np.log2(L) * 2.0 ** -24 * pair)


def test_rejected_plans(fd):
    for args in [(10.0, 16, 16, 16, 8, 1, 1),     # source inside the volume
                 (64.0, 16, 8200, 16, 8, 1, 1),   # detector wider than the filter takes
                 (64.0, 16, 16, 16, 8, 1, 3)]:    # D does not divide P
        with pytest.raises(fd.FdkodError) as e:
            fd.Plan(*args)
        assert e.value.status == -2


def test_out_of_memory_plan_fails_cleanly(fd):
    """A plan whose decomposed-data workspace cannot exist (s = 0, 32768
    detector rows, ~10^14 bytes) returns FDKOD_ERR_OOM, frees what it had
    allocated, and the library keeps working."""
    with pytest.raises(fd.FdkodError) as e:
        fd.Plan(4.0 * 2048, 2048, 2048, 32768, 2048, 0, 2)
    assert e.value.status == -4
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        with pytest.raises(fd.FdkodError):
            fd.Plan(4.0 * 2048, 2048, 2048, 32768, 2048, 0, 2)
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < 64 << 20          # nothing left behind
    N, P = 32, 48
    Q = torch.from_numpy(np.random.default_rng(830).standard_normal((P, N, N)).astype(np.float32)).cuda()
    with fd.Plan(4.0 * N, N, N, N, P, 2, 4) as plan:
        plan.backproject(Q)
        assert plan.device_status() == 0


def test_concurrent_plans_on_two_streams(fd):
    """Two plans (different geometries) enqueued on two streams at once give
    the same volumes as one after the other."""
    rng = np.random.default_rng(840)
    Qa = torch.from_numpy(rng.standard_normal((96, 64, 64)).astype(np.float32)).cuda()
    Qb = torch.from_numpy(rng.standard_normal((60, 50, 53)).astype(np.float32)).cuda()
    with fd.Plan(256.0, 64, 64, 64, 96, 3, 4) as pa, fd.Plan(200.0, 50, 53, 50, 60, 2, 3) as pb:
        ref_a = pa.backproject(Qa).clone()
        ref_b = pb.backproject(Qb).clone()
        torch.cuda.synchronize()
        sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
        va = torch.empty_like(ref_a)
        vb = torch.empty_like(ref_b)
        for _ in range(3):
            pa.backproject(Qa, va, sa.cuda_stream)
            pb.backproject(Qb, vb, sb.cuda_stream)
        torch.cuda.synchronize()
        assert torch.equal(va, ref_a) and torch.equal(vb, ref_b)
        assert pa.device_status() == 0 and pb.device_status() == 0


def test_wrong_tensors_are_refused_before_launch(fd):
    """Tensors of the wrong shape, dtype or layout never reach the library:
    the binding raises ValueError and the plan stays usable."""
    N, P, s, D = 32, 48, 1, 4
    with fd.Plan(4.0 * N, N, N, N, P, s, D) as plan:
        Q = torch.zeros((P, N, N), device="cuda")
        vol = torch.empty((N, N, N), device="cuda")
        bad = [lambda: plan.filter(torch.zeros((P, N, N - 1), device="cuda")),
               lambda: plan.filter(torch.zeros((P, N, N), dtype=torch.float64, device="cuda")),
               lambda: plan.backproject(torch.zeros((P - 1, N, N), device="cuda")),
               lambda: plan.backproject(Q, torch.empty((N, N, N - 1), device="cuda")),
               lambda: plan.backproject(Q.transpose(1, 2)),
               lambda: plan.backproject(Q.cpu()),
               lambda: plan.decompose(Q, torch.empty(8, device="cuda")),
               lambda: plan.backproject_decomposed(torch.empty(8, device="cuda"), vol),
               lambda: plan.net_backward(Q, torch.zeros(1439, device="cuda"),
                                         torch.zeros(plan.decomposed_shape, device="cuda"), 0, N,
                                         torch.zeros(1440, device="cuda"))]
        for f in bad:
            with pytest.raises(ValueError):
                f()
        plan.backproject(Q, vol)
        torch.cuda.synchronize()
        assert plan.device_status() == 0
        assert float(vol.abs().max()) == 0.0
