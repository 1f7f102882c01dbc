"""Piecemeal (slab-wise) reconstruction, Sec. 2.2: each slab reads only the
detector rows the b formula says it needs.  Slab-wise output must equal the
whole-volume output and the oracle to the parity bar, bands that miss needed
rows must be rejected, and the device memory must shrink."""
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


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("N,P,s,D,slab,qtype", [(64, 96, 3, 4, 16, "f32"), (48, 60, 2, 1, 32, "f32"),
                                                 (64, 96, 2, 4, 32, "bf16")])
def test_slabs_equal_whole_volume_and_oracle(fd, oracle_mod, N, P, s, D, slab, qtype):
    R = 4.0 * N
    p = phantom.project(phantom.make_phantom(900 + N, N, 8), R, N, N, P)
    with fd.Plan(R, N, N, N, P, s, D, qtype=qtype) as full:
        whole = full.backproject(full.filter(torch.from_numpy(p).cuda())).cpu().numpy()
    with fd.Plan(R, N, N, N, P, s, D, qtype=qtype, workspace=False) as plan:
        got = fd.reconstruct_slabs(plan, p, slab)
        assert plan.device_status() == 0
    assert _rel(got, whole) <= 1e-5
    if qtype == "f32":
        want = oracle_mod.fdkod(oracle_mod.filter(p, R), R, N, s, D)
        assert _rel(got, want) <= 1e-5


def test_band_must_cover_the_slab(fd):
    N, P = 64, 96
    with fd.Plan(4.0 * N, N, N, N, P, 3, 4, workspace=False) as plan:
        z0, nz = 48, 16
        v0, nr = plan.slab_rows(z0, nz)
        assert 0 <= v0 and v0 + nr <= N and nr >= nz
        Q = torch.zeros((P, nr - 2, N), device="cuda")
        S = torch.empty(plan.slab_workspace_elems(nr), device="cuda")
        with pytest.raises(fd.FdkodError) as e:
            plan.backproject_slab(Q, v0 + 2, S, z0, nz)
        assert e.value.status == -1
        with pytest.raises(fd.FdkodError):
            plan.backproject(torch.zeros((P, N, N), device="cuda"))   # no whole-volume workspace


def test_streaming_uses_far_less_device_memory(fd):
    N, P, s, D = 256, 360, 2, 4
    R = 4.0 * N
    p = phantom.project(phantom.make_phantom(950, N, 10), R, N, N, P)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    base = torch.cuda.memory_allocated()
    with fd.Plan(R, N, N, N, P, s, D) as full:
        whole = full.backproject(full.filter(torch.from_numpy(p).cuda())).cpu().numpy()
        torch.cuda.synchronize()
        full_peak = torch.cuda.max_memory_allocated() - base + full.info["device_bytes"]
    with fd.Plan(R, N, N, N, P, s, D, workspace=False) as plan:
        got = fd.reconstruct_slabs(plan, p, 32)
        slab_peak = plan.info["device_bytes"] + plan.last_slab_device_bytes
    assert slab_peak < 0.5 * full_peak, (slab_peak, full_peak)
    assert _rel(got, whole) <= 1e-5


def test_pinned_torch_buffers_and_ragged_last_slab(fd):
    """Page-locked torch host tensors in and out; a slab size that leaves a
    short last slab; two runs in a row give the same volume."""
    N, P, s, D = 72, 96, 2, 4
    R = 4.0 * N
    p = phantom.project(phantom.make_phantom(960, N, 8), R, N, N, P)
    src = torch.from_numpy(p).pin_memory()
    out = torch.empty((N, N, N), dtype=torch.float32).pin_memory()
    with fd.Plan(R, N, N, N, P, s, D) as full:
        whole = full.backproject(full.filter(src.cuda())).cpu().numpy()
    with fd.Plan(R, N, N, N, P, s, D, workspace=False) as plan:
        fd.reconstruct_slabs(plan, src, 20, out)          # slabs of 20, 20, 20, 12
        first = out.clone()
        fd.reconstruct_slabs(plan, src, 20, out)
        assert plan.device_status() == 0
    assert torch.equal(first, out)
    assert _rel(out.numpy(), whole) <= 1e-5
