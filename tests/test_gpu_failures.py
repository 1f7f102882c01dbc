"""Device-side failure reporting, exercised without a GPU fault.

The staged backprojection waits on its copies with a wall-clock limit and
checks every staging window before reading it.  The plan's test hook
(fdkod_set_test_fault) drives both paths on purpose: one CTA leaves out one
copy, so its bounded wait (here 20 ms) runs out and the kernel reports
FDKOD_ERR_TIMEOUT after waiting for its other copies; or every window counts
as too small, so every view is skipped (nothing is read outside a window)
and FDKOD_ERR_BOUNDS is reported.  Afterwards the same plan, with the hook
cleared, must again match the oracle: the context stays usable."""
import numpy as np
import pytest

import phantom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_RMSE = 1e-5
MAX_REL = 2e-4
WAIT_NS = 20_000_000  # 20 ms


@pytest.fixture(scope="module")
def fd():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1708_07515_gb300 as fd
    fd.load()
    return fd


def _case(oracle_mod, N=64, P=64):
    R = 4.0 * N
    p = phantom.project(phantom.make_phantom(4100 + N, N, 8), R, N, N, P)
    Q = oracle_mod.filter(p, R).astype(np.float32)
    return R, Q


def _cmp(got, want, what):
    err = got.astype(np.float64) - want
    rel = np.linalg.norm(err) / np.linalg.norm(want)
    mx = np.abs(err).max() / np.abs(want).max()
    assert rel <= REL_RMSE and mx <= MAX_REL, f"{what}: rel-RMSE {rel:.3e}, max-rel {mx:.3e}"


@pytest.mark.parametrize("D", [1, 2])
def test_a_copy_that_never_lands_reports_timeout(fd, oracle_mod, D):
    N, P, s = 64, 64, 1
    R, Q = _case(oracle_mod, N, P)
    Qd = torch.from_numpy(Q).cuda()
    with fd.Plan(R, N, N, N, P, s, D) as plan:
        w, _ = plan.tile
        assert w > 0, "the staged (TMA) kernel must be the one that runs"
        fd.fdkod_set_test_fault(plan.handle, fd.FDKOD_TEST_SKIP_COPY, WAIT_NS)
        plan.backproject(Qd)
        torch.cuda.synchronize()
        assert plan.device_status() == -5   # FDKOD_ERR_TIMEOUT
        assert plan.device_status() == 0    # read and cleared
        fd.fdkod_set_test_fault(plan.handle, fd.FDKOD_TEST_NONE, 0)
        got = plan.backproject(Qd).cpu().numpy()
        assert plan.device_status() == 0
    _cmp(got, oracle_mod.fdkod(Q, R, N, s, D), f"after the timeout, D={D}")


def test_an_undersized_window_reports_bounds_and_reads_nothing(fd, oracle_mod):
    N, P, s, D = 64, 64, 2, 4
    R, Q = _case(oracle_mod, N, P)
    Qd = torch.from_numpy(Q).cuda()
    with fd.Plan(R, N, N, N, P, s, D) as plan:
        fd.fdkod_set_test_fault(plan.handle, fd.FDKOD_TEST_SMALL_WINDOW, WAIT_NS)
        vol = plan.backproject(Qd)
        assert plan.device_status() == -6   # FDKOD_ERR_BOUNDS
        # every view was skipped: nothing accumulated
        assert float(vol.abs().max()) == 0.0
        fd.fdkod_set_test_fault(plan.handle, fd.FDKOD_TEST_NONE, 0)
        got = plan.backproject(Qd).cpu().numpy()
        assert plan.device_status() == 0
    _cmp(got, oracle_mod.fdkod(Q, R, N, s, D), "after the window overflow")


def test_the_hook_rejects_unknown_kinds(fd):
    with fd.Plan(256.0, 64, 64, 64, 8, 1, 2) as plan:
        for kind, wait in ((3, 0), (-1, 0), (1, -5)):
            with pytest.raises(fd.FdkodError):
                fd.fdkod_set_test_fault(plan.handle, kind, wait)
