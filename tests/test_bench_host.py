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
