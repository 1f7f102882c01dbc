"""Host logic of bench.py that needs no GPU: the DRAM-traffic record of the
backprojection kernel is reported only for the workload it was taken on and
only while the kernel's source text is the one that was profiled."""
import os
import shutil

import bench


def test_traffic_record_applies_to_its_own_workload_only():
    got = bench.recorded_bp_traffic("fdkod_512")
    assert isinstance(got, int) and got > 0
    assert bench.recorded_bp_traffic("fdkod_1024") is None


def test_traffic_record_is_dropped_once_the_kernel_text_changes(tmp_path, monkeypatch):
    root = bench.ROOT
    os.makedirs(tmp_path / "profiles")
    os.makedirs(tmp_path / "paper_1708_07515_gb300" / "csrc")
    shutil.copy(os.path.join(root, "profiles", "dram_traffic_fdkod_512.md"), tmp_path / "profiles")
    src = open(os.path.join(root, "paper_1708_07515_gb300", "csrc", "backproject.cu")).read()
    dst = tmp_path / "paper_1708_07515_gb300" / "csrc" / "backproject.cu"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    dst.write_text(src)
    assert bench.recorded_bp_traffic("fdkod_512") is not None
    # text outside the kernel may change
    dst.write_text(src + "\n// trailing comment\n")
    assert bench.recorded_bp_traffic("fdkod_512") is not None
    # one changed statement inside it may not
    i = src.index("template <typename TS, bool DIRECT, int WD>\n__global__")
    j = src.index("\n}\n", i)
    body = src[i:j]
    assert "acc[i] * a.scale" in body
    dst.write_text(src[:i] + body.replace("acc[i] * a.scale", "acc[i] * a.scale * 1.0f", 1) + src[j:])
    assert bench.recorded_bp_traffic("fdkod_512") is None


def _run_bench(args, env_extra=None):
    import subprocess
    import sys
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py")] + args, cwd=bench.ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference times the oracle on the host cores (no GPU)
    and prints one JSON line with the keys of the bench contract."""
    import json
    r = _run_bench(["--impl", "reference", "--workload", "fdkod_128", "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["unit"] == "voxel-updates/s" and j["higher_is_better"] is True
    assert j["value"] > 0 and j["steps"] == 1 and j["warmup"] == 3
    assert j["config"]["workload"] == "fdkod_128^3_P128_s2_D2"
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == j["value"] and cb["cores"] >= 1 and cb["sample"]
    assert j["e2e"] == {"value": j["value"], "unit": j["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    r = _run_bench(["--impl", "reference", "--workload", "fdkod_128", "--steps", "1", "--warmup", "3"],
                   {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""
