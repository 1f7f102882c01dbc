"""Host logic of bench.py that needs no GPU: the DRAM-traffic record of the
backprojection kernel is reported only for the workload it was taken on and
only while the kernel's source text is the one that was profiled."""
import os
import shutil

import bench


KERNEL_LINE = "template <typename TS, bool DIRECT, int WD>"


def _tree(tmp_path, monkeypatch, src, workload="fdkod_512"):
    """A copy of the two files the record reads, with a record whose hash
    matches the kernel text of `src` (as a fresh capture would write it)."""
    import hashlib
    os.makedirs(tmp_path / "profiles", exist_ok=True)
    os.makedirs(tmp_path / "paper_1708_07515_gb300" / "csrc", exist_ok=True)
    dst = tmp_path / "paper_1708_07515_gb300" / "csrc" / "backproject.cu"
    dst.write_text(src)
    sha = hashlib.sha256(bench.kernel_text(src, KERNEL_LINE).encode()).hexdigest()
    (tmp_path / bench.TRAFFIC_PROFILE).write_text(
        "# summary\n\nbp_traffic_bytes_per_launch: 123456\n"
        f"bp_traffic_workload: {workload}\nbp_traffic_source: backproject.cu\n"
        f"bp_traffic_kernel_first_line: {KERNEL_LINE}\nbp_traffic_kernel_sha256: {sha}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return dst


def _src():
    return open(os.path.join(bench.ROOT, "paper_1708_07515_gb300", "csrc", "backproject.cu")).read()


def test_committed_record_names_its_kernel():
    text = open(os.path.join(bench.ROOT, bench.TRAFFIC_PROFILE)).read()
    fields = dict(l.split(": ", 1) for l in text.splitlines() if l.startswith("bp_traffic_"))
    src = open(os.path.join(bench.ROOT, "paper_1708_07515_gb300", "csrc", fields["bp_traffic_source"])).read()
    assert bench.kernel_text(src, fields["bp_traffic_kernel_first_line"])
    assert int(fields["bp_traffic_bytes_per_launch"]) > 0


def test_traffic_record_applies_to_its_own_workload_only(tmp_path, monkeypatch):
    _tree(tmp_path, monkeypatch, _src())
    assert bench.recorded_bp_traffic("fdkod_512") == 123456
    assert bench.recorded_bp_traffic("fdkod_1024") is None


def test_traffic_record_is_dropped_once_the_kernel_text_changes(tmp_path, monkeypatch):
    src = _src()
    dst = _tree(tmp_path, monkeypatch, src)
    assert bench.recorded_bp_traffic("fdkod_512") is not None
    # text outside the kernel may change
    dst.write_text(src + "\n// trailing comment\n")
    assert bench.recorded_bp_traffic("fdkod_512") is not None
    # one changed statement inside it may not
    body = bench.kernel_text(src, KERNEL_LINE)
    assert "acc[i] * a.scale" in body
    dst.write_text(src.replace(body, body.replace("acc[i] * a.scale", "acc[i] * a.scale * 1.0f", 1)))
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


def test_stage_rooflines_count_compulsory_and_crop_bytes():
    """The streaming stages' bytes: the filter reads the projections and
    writes Q; the decomposition reads Q once and writes S' once, and its crop
    reads are every square's T_q + 1 columns of every row and view."""
    import types
    w = types.SimpleNamespace(P=8, Nv=4, Nu=16, D=2)
    info = {"decomposed_elems": 1000}
    T = [10, 12, 9]
    r = bench.stage_rooflines(w, info, {"filter": 1.0, "decompose": 2.0}, "bf16", {"hbm_gbs": 1000.0}, T=T)
    samples = 8 * 4 * 16
    assert r["filter"]["bytes"] == samples * (4 + 2)
    assert r["decompose"]["bytes"] == samples * 2 + 1000 * 4
    assert r["decompose"]["crop_read_bytes"] == (11 + 13 + 10) * 4 * 8 * 2
    assert abs(r["decompose"]["crop_read_frac"] - r["decompose"]["crop_read_bytes"] / 2e-3 / 1e9 / 1000.0) < 1e-12
    assert r["peak_note"] == "measured copy bandwidth"
    assert "crop_read_bytes" not in bench.stage_rooflines(w, info, {"filter": 1.0, "decompose": 2.0}, "f32", {})[
        "decompose"]
