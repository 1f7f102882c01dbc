"""The allocation-free backprojection entry point (fdkod_backproject_noalloc).

It serves callers that cannot call cudaMalloc (memory fixed at start-up, or
a device already reserved by another pool): all of its working memory sits
in one fixed device array inside the library.  Called through the C ABI, its
output must match the planned entry point (fdkod_plan + fdkod_backproject)
to the parity tolerance, on consecutive calls that reuse the same array.
This file is collected last on purpose.
"""
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


def _case(oracle_mod, N, P, seed):
    R = 4.0 * N
    p = phantom.project(phantom.make_phantom(seed, N, 8), R, N, N, P)
    return R, torch.from_numpy(oracle_mod.filter(p, R).astype(np.float32)).cuda()


def _close(got, want):
    g = got.double()
    w = want.double().to(g.device)
    rel = float(torch.linalg.norm(g - w) / torch.linalg.norm(w))
    mx = float((g - w).abs().max() / w.abs().max())
    assert rel <= REL_RMSE and mx <= MAX_REL, (rel, mx)


def test_noalloc_matches_planned_backprojection(fd, oracle_mod):
    cases = [(128, 128, 2, 2, 3001), (64, 96, 3, 4, 3002), (48, 48, 2, 1, 3003)]
    refs = []
    for N, P, s, D, seed in cases:
        R, Q = _case(oracle_mod, N, P, seed)
        with fd.Plan(R, N, N, N, P, s, D) as plan:
            refs.append((R, N, P, s, D, Q, plan.backproject(Q).clone()))
    torch.cuda.synchronize()
    # two calls in a row on the same geometry, then other geometries, then the
    # first again: each call must not depend on what the previous one left
    order = [0, 0, 1, 2, 0]
    for i in order:
        R, N, P, s, D, Q, want = refs[i]
        vol = torch.full((N, N, N), float("nan"), device="cuda")
        fd.fdkod_backproject_noalloc(R, N, N, N, P, s, D, Q, vol)
        assert fd.fdkod_noalloc_device_status() == 0
        _close(vol, want)


@pytest.mark.parametrize("N,P,s,D,Rf", [(64, 96, 3, 4, 4.0), (48, 60, 2, 3, 1.3), (40, 32, 1, 2, 0.9),
                                        (33, 48, 3, 6, 2.0), (96, 72, 2, 8, 4.0)])
def test_noalloc_matches_the_oracle(fd, oracle_mod, N, P, s, D, Rf):
    """Directly against the FP64 oracle's FDK-OD, over decomposition levels,
    ragged squares and short source distances; the status word also says
    the host bound of the shifted-row width held (FDKOD_OK, not BOUNDS)."""
    R = max(Rf * N, np.sqrt(2.0) * N / 2 + 1.5)
    p = phantom.project(phantom.make_phantom(3100 + N, N, 8), R, N, N, P)
    Q = oracle_mod.filter(p, R).astype(np.float32)
    vol = torch.full((N, N, N), float("nan"), device="cuda")
    fd.fdkod_backproject_noalloc(R, N, N, N, P, s, D, torch.from_numpy(Q).cuda(), vol)
    assert fd.fdkod_noalloc_device_status() == 0
    _close(vol, torch.from_numpy(oracle_mod.fdkod(Q, R, N, s, D)).cuda())


def test_noalloc_rejects_problems_over_its_fixed_memory(fd):
    N, P = 512, 720
    Q = torch.zeros((P, N, N), device="cuda")
    vol = torch.zeros((N, N, N), device="cuda")
    with pytest.raises(fd.FdkodError) as e:
        fd.fdkod_backproject_noalloc(4.0 * N, N, N, N, P, 3, 4, Q, vol)
    assert e.value.status == -2
