"""Whole reconstruction from host buffers (fdkod_reconstruct): projections
in host memory, volume in host memory, the copies overlapped with the
filter and the backprojection inside the call.  It runs the same kernels as
the device-buffer entry points, in bands of detector rows (filter,
decomposition) and groups of slices (backprojection) that keep their operand
pairings, so its volume equals fdkod_filter + fdkod_backproject bit for bit
(even Nv); and it meets the FP64 oracle at the parity bar."""
import numpy as np
import pytest

import phantom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1708_07515_gb300 as fd
    fd.load()
    return fd


@pytest.mark.parametrize("N,P,s,D,qtype", [(96, 120, 2, 4, "f32"), (70, 90, 1, 3, "f32"), (64, 64, 0, 1, "f32"),
                                            (128, 96, 2, 2, "bf16")])
def test_host_buffer_reconstruction_equals_the_device_path(fd, oracle_mod, N, P, s, D, qtype):
    R = 4.0 * N
    proj = phantom.project(phantom.make_phantom(5200 + N, N, 10), R, N, N, P)
    with fd.Plan(R, N, N, N, P, s, D, qtype=qtype) as plan:
        want = plan.backproject(plan.filter(torch.from_numpy(proj).cuda())).cpu().numpy()
        pinned = torch.from_numpy(proj).pin_memory()
        out = torch.empty((N, N, N), dtype=torch.float32).pin_memory()
        for _ in range(2):  # the second call reuses the plan's buffers
            out.fill_(float("nan"))
            fd.reconstruct(plan, pinned, out)
            assert np.array_equal(out.numpy(), want)
        # pageable host memory works too
        got = fd.reconstruct(plan, proj)
        assert np.array_equal(got, want)
        assert plan.info["device_bytes"] > 0
    if qtype == "f32":
        ref = oracle_mod.fdkod(oracle_mod.filter(proj, R), R, N, s, D)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= 1e-5, rel


@pytest.mark.parametrize("offset", [0, 1, 4])
def test_host_buffer_inside_a_larger_page_locked_allocation(fd, offset):
    """Projections at an offset inside a bigger page-locked buffer: from a
    16-byte aligned start the call reads its first bands straight from the
    buffer (the allocation covers the projections), from a 4-byte offset it
    copies every band through the copy engine; both give the device path's
    volume bit for bit."""
    N, P, s, D = 64, 72, 1, 2
    R = 4.0 * N
    proj = phantom.project(phantom.make_phantom(5250, N, 8), R, N, N, P)
    big = torch.zeros(proj.size + 8, dtype=torch.float32).pin_memory()
    view = big[offset:offset + proj.size].view(P, N, N)
    view.copy_(torch.from_numpy(proj))
    with fd.Plan(R, N, N, N, P, s, D) as plan:
        want = plan.backproject(plan.filter(torch.from_numpy(proj).cuda())).cpu().numpy()
        got = fd.reconstruct(plan, view)
    assert np.array_equal(got, want)


def test_host_buffer_reconstruction_with_an_odd_detector_height(fd, oracle_mod):
    """Nv odd: one band of rows (the filter's row pairs then match the
    whole-detector launch's only up to FFT round-off)."""
    N, Nu, Nv, P, s, D = 48, 52, 47, 60, 2, 3
    R = 4.0 * N
    proj = phantom.project(phantom.make_phantom(5300, N, 8), R, Nu, Nv, P)
    with fd.Plan(R, N, Nu, Nv, P, s, D) as plan:
        want = plan.backproject(plan.filter(torch.from_numpy(proj).cuda())).cpu().numpy()
        got = fd.reconstruct(plan, proj)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-6
    ref = oracle_mod.fdkod(oracle_mod.filter(proj, R), R, N, s, D)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5


def test_host_buffer_reconstruction_needs_the_workspace(fd):
    with fd.Plan(256.0, 64, 64, 64, 32, 1, 2, workspace=False) as plan:
        with pytest.raises(fd.FdkodError) as e:
            fd.reconstruct(plan, np.zeros((32, 64, 64), np.float32))
        assert e.value.status == -1
