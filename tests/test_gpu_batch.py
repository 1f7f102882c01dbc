"""Batched reconstruction of volumes of uneven size in one CUDA graph, against
eager launches (bit for bit) and against the FP64 oracle (parity bar); the
persistent batched backprojection against each plan's own launch."""
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


def test_graph_batch_matches_eager_and_oracle(fd, oracle_mod):
    from paper_1708_07515_gb300.batch import BatchReconstructor, Instance
    sizes = (32, 40, 48, 64)
    work = phantom.batched_workload(seed=4100, count=6, sizes=sizes, n_ell=6)
    insts = [Instance(R, N, N, N, P) for N, P, R, _ in work]
    projs = [phantom.project(phantom.make_phantom(sd, N, 6), R, N, N, P) for N, P, R, sd in work]
    br = BatchReconstructor(insts, rates=(1.5e12, 4e11))
    try:
        for inst in insts:
            assert inst.P % inst.D == 0 and 0 <= inst.s <= 7
        br.load(projs)
        br.run_eager()
        torch.cuda.synchronize()
        eager = [v.clone() for v in br.vol]
        for v in br.vol:
            v.fill_(float("nan"))
        br.capture()
        br.replay()
        torch.cuda.synchronize()
        for a, b in zip(eager, br.vol):
            assert torch.equal(a, b)
        for inst, p, v in zip(insts, projs, br.vol):
            Q = oracle_mod.filter(p, inst.R)
            want = oracle_mod.fdkod(Q, inst.R, inst.N, inst.s, inst.D)
            got = v.cpu().numpy().astype(np.float64)
            rel = np.linalg.norm(got - want) / np.linalg.norm(want)
            assert rel <= 1e-5, (inst, rel)
        assert all(p.device_status() == 0 for p in br.plans)
    finally:
        br.close()


@pytest.mark.parametrize("persistent", [True, False])
def test_persistent_batch_equals_per_plan_launches(fd, oracle_mod, persistent):
    """The batch graph's per-volume branches give each volume bit for bit
    what its own backprojection launch gives.  The persistent kernel (one
    launch, work list over volumes, tiles and z-slabs of 32 slices; plans
    with D = 1 read Q, the others their workspace) evaluates the same sums
    with the row coordinate in float32 where the per-volume launch (slice
    pairs) uses fixed point: equal to float32 rounding."""
    from paper_1708_07515_gb300.batch import BatchReconstructor, Instance
    insts = [Instance(4.0 * 48, 48, 48, 48, 64, 2, 4), Instance(4.0 * 40, 40, 44, 36, 60, 0, 1),
             Instance(4.0 * 64, 64, 64, 64, 90, 3, 3), Instance(4.0 * 33, 33, 36, 40, 48, 1, 2)]
    projs = [phantom.project(phantom.make_phantom(4200 + k, i.N, 6), i.R, i.Nu, i.Nv, i.P)
             for k, i in enumerate(insts)]
    br = BatchReconstructor(insts, streams=3, persistent=persistent)
    try:
        assert (br.batch is not None) == persistent
        br.load(projs)
        br.capture()
        br.replay()
        torch.cuda.synchronize()
        for inst, plan, Q, v in zip(insts, br.plans, br.Q, br.vol):
            ref = plan.backproject(Q)
            torch.cuda.synchronize()
            if persistent:
                d = (v.double() - ref.double())
                assert float(d.norm() / ref.double().norm()) <= 1e-6, inst
                assert float(d.abs().max() / ref.abs().max()) <= 2e-5, inst
            else:
                assert torch.equal(v, ref), inst
            assert plan.device_status() == 0
        # and against the oracle (parity bar)
        for inst, p, v in zip(insts, projs, br.vol):
            Q = oracle_mod.filter(p, inst.R).astype(np.float32)
            want = oracle_mod.fdkod(Q, inst.R, inst.N, inst.s, inst.D)
            got = v.cpu().numpy().astype(np.float64)
            assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-5, inst
        assert br.launches() == sum(3 if i.D > 1 else 2 for i in insts) + (1 if persistent else len(insts))
    finally:
        br.close()


def test_measured_rates_are_positive(fd):
    from paper_1708_07515_gb300 import autotune
    bp, dec = autotune.measure_rates(N=64, P=60)
    assert bp > 1e9 and dec > 1e8


def test_gpu_projector_matches_cpu_projector(fd):
    """Input generation for large workloads: the GPU projector (FP32) agrees
    with the FP64 CPU projector."""
    N, P = 96, 24
    R = 4.0 * N
    ell = phantom.make_phantom(4242, N, 20)
    cpu = phantom.project(ell, R, N + 4, N - 6, P, dtype=np.float64)
    gpu = phantom.project_gpu(ell, R, N + 4, N - 6, P).cpu().numpy().astype(np.float64)
    assert np.abs(gpu - cpu).max() <= 2e-5 * np.abs(cpu).max()


def test_batch_create_rejects_what_it_cannot_take(fd):
    """A plan with 16-bit Q and D = 1 (16-bit windows) and a decimating plan
    without a workspace are refused; the refusal leaves the plans usable."""
    vol = torch.empty((32, 32, 32), device="cuda")
    Q16 = torch.zeros((48, 32, 32), dtype=torch.bfloat16, device="cuda")
    with fd.Plan(128.0, 32, 32, 32, 48, 1, 1, qtype="bf16") as p16, \
            fd.Plan(128.0, 32, 32, 32, 48, 1, 4, workspace=False) as pnw:
        with pytest.raises(fd.FdkodError) as e:
            fd.BatchBackprojection([p16], [Q16], [vol])
        assert e.value.status == -2
        with pytest.raises(fd.FdkodError) as e:
            fd.BatchBackprojection([pnw], [None], [vol])
        assert e.value.status == -1
        p16.backproject(Q16, vol)
        assert p16.device_status() == 0


def test_tile_width_choice_keeps_results(fd):
    """Every valid staging-window width gives the same volume bit for bit;
    too narrow or uninstantiated widths are refused; the autotuner's choice
    is one of the candidates and stays set on the plan."""
    from paper_1708_07515_gb300 import autotune
    N, P = 64, 90
    R = 4.0 * N
    Q = torch.from_numpy(np.random.default_rng(4300).standard_normal((P, N, N)).astype(np.float32)).cuda()
    for s, D in ((2, 3), (1, 1)):
        with fd.Plan(R, N, N, N, P, s, D) as plan:
            cur, narrowest = plan.tile
            assert cur == narrowest > 0
            ref = plan.backproject(Q).clone()
            for w in autotune.tile_candidates(narrowest, count=5):
                plan.set_tile(w)
                assert plan.tile[0] == w
                assert torch.equal(plan.backproject(Q), ref), (s, D, w)
            for bad in (narrowest - 16, 40):
                if bad > 0 and bad not in autotune.TILE_WIDTHS or bad < narrowest:
                    with pytest.raises(fd.FdkodError):
                        plan.set_tile(bad)
            plan.set_tile(0)
            assert plan.tile[0] == narrowest
            best, times = autotune.choose_tile(plan)
            assert best in times and plan.tile[0] == best
            assert torch.equal(plan.backproject(Q), ref)
            assert plan.device_status() == 0
