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
    w = want.double()
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
        torch.cuda.synchronize()
        _close(vol, want)


def test_noalloc_rejects_problems_over_its_fixed_memory(fd):
    N, P = 512, 720
    Q = torch.zeros((P, N, N), device="cuda")
    vol = torch.zeros((N, N, N), device="cuda")
    with pytest.raises(fd.FdkodError) as e:
        fd.fdkod_backproject_noalloc(4.0 * N, N, N, N, P, 3, 4, Q, vol)
    assert e.value.status == -2
