#!/usr/bin/env python
"""Benchmark of the FDK-OD hot path on GB300.

One step = one pass of the whole path over one synthetic scan: the FP64
bound kernel (Eq. 1 at square vertices), the FFT ramp filter, the
decomposition (shift + angular decimation) and the per-square
backprojection.  Workload: 512^3 volume from 720 views of a 512^2 detector,
s = 3, D = 4, 40 seeded random ellipsoids + 1 % Gaussian noise (synthetic
stand-in for the paper's phantom and scanner data).

Metric: effective voxel-updates/s = N^3 P / t_step (the plain-FDK-equivalent
work; FDK-OD performs N^3 P / D updates).  The plain FDK baseline runs the
same filter plus the plain backprojection on the same GPU.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank reconstructs its own independent scan (weak
scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FDK-OD voxel-updates/s vs plain FDK on one GB300 at fixed RMSE vs FP64 oracle"
UNIT = "voxel-updates/s"
WORKLOAD_KEY = "fdkod_512"
# Algorithmic FP32 operations per voxel update of the backprojection, one
# issue slot each (an FMA is one operation): row coordinate (FMA), floor,
# fraction, three lerps (subtract + FMA each), weighted accumulate (FMA)
OPS_PER_UPDATE = 10
# the same work counted as FLOPs (FMA = 2) against the FMA peak
FLOP_PER_UPDATE = 14
# on-chip bytes per update: the four float32 samples of the bilinear gather
SMEM_BYTES_PER_UPDATE = 16
FP32_LANES_PER_SM = 128
SMEM_BYTES_PER_CLK_PER_SM = 128


def sm_count(device=0) -> int:
    """Streaming multiprocessors of the device the bench runs on."""
    import torch
    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def workload_config(w, qtype="f32", taps="triangle") -> dict:
    """The workload keys both arms' JSON lines carry."""
    return {"workload": w.name, "N": w.N, "P": w.P, "Nu": w.Nu, "Nv": w.Nv, "R": w.R, "s": w.s, "D": w.D,
            "q_storage": qtype, "taps": taps}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD_KEY)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffer) measurement")
    ap.add_argument("--batched", action="store_true",
                    help="64 volumes of uneven size (N in {64..384}, P = 1.4 N) in one CUDA graph")
    ap.add_argument("--persistent", action="store_true",
                    help="batched form: all volumes' backprojections in one persistent launch (after every "
                         "decomposition) instead of one launch per volume on its stream")
    ap.add_argument("--split", choices=["scans", "z"], default="scans",
                    help="with several ranks: each reconstructs its own scan (weak scaling), or one volume is split "
                         "into z-slabs, each rank holding only the detector rows its slab reads (strong scaling)")
    ap.add_argument("--slabs", type=int, default=0,
                    help="slab-wise (piecemeal, Sec. 2.2) reconstruction from host buffers, this many slices per slab")
    ap.add_argument("--qtype", choices=["f32", "bf16", "f16"], default="f32",
                    help="storage type of the filtered projections (arithmetic stays float32)")
    ap.add_argument("--taps", choices=["triangle", "sinc", "learned", "net"], default="triangle",
                    help="angular low-pass of the decomposition (Sec. 2.1): triangle, Hann-windowed sinc, taps "
                         "fitted to full FDK on separate training scans before the run (learn.py), or the triangle "
                         "plus the learned residual net (three tensor-core layers; weights from --net-weights)")
    ap.add_argument("--net-weights", default=None,
                    help="weights of the learned decimation (.npy, 1440 values, learn_net.py --out); default: "
                         "the package's trained weights for this D if present, else seeded random weights")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def rows_for_slices(N, Nv, R, zs):
    """Detector rows the given slices can touch (b formula of Sec. 2.2 with
    U in [1 - r/R, 1 + r/R])."""
    rmax = math.sqrt(2.0) * 0.5 * (N - 1)
    vc = 0.5 * (Nv - 1)
    need = set()
    for zi in zs:
        z = zi - 0.5 * (N - 1)
        va, vb = z / (1 - rmax / R) + vc, z / (1 + rmax / R) + vc
        for r in range(int(math.floor(min(va, vb))) - 1, int(math.floor(max(va, vb))) + 3):
            if 0 <= r < Nv:
                need.add(r)
    return sorted(need)


def oracle_sample(w, proj, zs, oracle):
    """The FP64 oracle on a bounded sample: filter the rows the slices need
    (direct convolution), then FDK-OD on those slices.  Returns seconds."""
    rows = rows_for_slices(w.N, w.Nv, w.R, zs)
    flat = np.array([k * w.Nv + v for k in range(w.P) for v in rows], dtype=np.int64)
    t0 = time.perf_counter()
    Qr = oracle.filter_rows(proj, w.R, flat)
    Q = np.zeros((w.P, w.Nv, w.Nu), dtype=np.float64)
    Q.reshape(-1, w.Nu)[flat] = Qr
    oracle.fdkod_slices(Q, w.R, w.N, w.s, w.D, zs)
    return time.perf_counter() - t0


def oracle_sample_fdk(w, proj, zs, oracle):
    """The same bounded sample through the oracle's plain FDK.  Returns seconds."""
    rows = rows_for_slices(w.N, w.Nv, w.R, zs)
    flat = np.array([k * w.Nv + v for k in range(w.P) for v in rows], dtype=np.int64)
    t0 = time.perf_counter()
    Qr = oracle.filter_rows(proj, w.R, flat)
    Q = np.zeros((w.P, w.Nv, w.Nu), dtype=np.float64)
    Q.reshape(-1, w.Nu)[flat] = Qr
    oracle.fdk_slices(Q, w.R, w.N, zs)
    return time.perf_counter() - t0


def reference_arm(args):
    """The oracle as it stands, timed on the host cores: each step is a
    bounded sample (one central slice) of the workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import phantom
    oracle.build()
    w = phantom.WORKLOADS[args.workload]
    proj = phantom.make_projections(w)
    cores = oracle.max_threads()
    order = np.random.default_rng(w.seed).permutation(w.N)
    times = []
    for i in range(args.warmup + args.steps):
        t = oracle_sample(w, proj, [int(order[i % w.N])], oracle)
        if i >= args.warmup:
            times.append(t)
    per_step = sum(times) / len(times)
    value = w.N * w.N * w.P / per_step
    sample = (f"one seeded slice of {w.name} per step: FP64 direct-convolution filter of the rows it needs + "
              "FP64 FDK-OD of the slice")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {**workload_config(w), "step": "bounds + filter + decompose + backproject (FP64 oracle, "
                                                  "one seeded slice per step)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


TRAFFIC_PROFILE = os.path.join("profiles", "dram_traffic_fdkod_512.md")


def kernel_text(src: str, marker: str) -> str:
    """A kernel's source text: from its first line `marker` to the closing
    brace at the start of a line."""
    a = src.index(marker + "\n")
    return src[a:src.index("\n}\n", a) + 3]


def recorded_bp_traffic(workload: str):
    """DRAM bytes per backprojection launch from the committed ncu summary,
    or None when the summary is for another workload or the kernel's source
    text has changed since the counters were taken."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, TRAFFIC_PROFILE)).read()
        fields = dict(line.split(": ", 1) for line in text.splitlines() if line.startswith("bp_traffic_"))
        src = open(os.path.join(ROOT, "paper_1708_07515_gb300", "csrc", fields["bp_traffic_source"])).read()
        body = kernel_text(src, fields["bp_traffic_kernel_first_line"])
        if fields.get("bp_traffic_workload") != workload:
            return None
        if fields.get("bp_traffic_kernel_sha256") != hashlib.sha256(body.encode()).hexdigest():
            return None
        return int(fields["bp_traffic_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        return None


def stage_rooflines(w, info, stages, qtype, peaks, T=None):
    """HBM fractions of the two streaming stages: algorithmic bytes (every
    input read once, every output written once) over the stage's event time,
    against the measured copy bandwidth (fallback 6800 GB/s).  With the
    squares' shifted-row lengths T_q the decomposition also gets its crop
    reads: every square reads its own T_q + 1 columns of every detector row
    and view (sum over q of (T_q + 1) Nv P samples), most of them served from
    L2 since neighbouring squares' crops overlap."""
    hbm = peaks.get("hbm_gbs") or 6800.0
    qb = 4 if qtype == "f32" else 2
    samples = float(w.P) * w.Nv * w.Nu
    filt = samples * (4 + qb)                                   # projections in, Q out
    dec = samples * qb + info["decomposed_elems"] * 4.0         # Q in, S' out
    out = {}
    for name, b in (("filter", filt), ("decompose", dec)):
        ach = b / (stages[name] * 1e-3) / 1e9
        out[name] = {"bound": "hbm", "bytes": b, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm}
    if T is not None and stages.get("decompose", 0) > 0:
        crop = float(sum(int(t) + 1 for t in T)) * w.Nv * w.P * qb
        ach = crop / (stages["decompose"] * 1e-3) / 1e9
        out["decompose"].update({"crop_read_bytes": crop, "crop_read_achieved": ach, "crop_read_frac": ach / hbm,
                                 "crop_read_note": "sum over squares of (T_q + 1) columns x Nv rows x P views "
                                                   "read, against the same peak (mostly L2 hits)"})
    out["peak_note"] = "measured copy bandwidth" if peaks.get("hbm_gbs") else "fallback 6800 GB/s"
    return out


def net_weights(path, D, seed=11):
    """(weights, source, base taps or None) of the learned decimation for
    --taps net; the base taps (the plain low-pass under the net) sit beside
    the weights as <name>_taps.npy when the net was trained on top of
    learned linear taps, else the base is the triangle."""
    if path is None:
        cand = os.path.join(ROOT, "paper_1708_07515_gb300", "net_weights", f"D{D}.npy")
        if os.path.exists(cand):
            path = cand
    if path is not None:
        tp = path[:-4] + "_taps.npy" if path.endswith(".npy") else path + "_taps.npy"
        base = np.load(tp).astype(np.float64) if os.path.exists(tp) else None
        return np.load(path).astype(np.float32), os.path.relpath(path, ROOT), base
    rng = np.random.default_rng(seed)
    w = np.concatenate([rng.standard_normal(80) * 0.4, rng.standard_normal(1280) * 0.15,
                        rng.standard_normal(80) * 0.01]).astype(np.float32)
    return w, f"seeded random weights (seed {seed}; throughput does not depend on the values)", None


def net_roofline(w, info, T, stages, peaks):
    """The learned decimation kernel, algorithmic work per launch: on the
    tensor cores layers 1 and 2 at every full-rate shifted sample (80 + 1280
    multiply-adds) and layer 3 at every decimated output (80); on the CUDA
    cores the shift interpolation (one lerp per sample) and the plain
    low-pass (2D - 1 taps per output).  Against the measured sustained dense
    BF16 peak and the derived FP32 peak."""
    samples = float(np.sum(T)) * w.Nv * w.P                 # full-rate shifted samples (T_q per square)
    outs = float(np.sum(T)) * w.Nv * (w.P // w.D)
    mma_flop = 2.0 * (1360.0 * samples + 80.0 * outs)
    fp32_flop = 2.0 * samples + 2.0 * (2 * w.D - 1) * outs
    t = stages["decompose"] * 1e-3
    bf16 = peaks.get("bf16_tflops_sustained") or 1700.0
    max_mhz = peaks.get("sm_max_mhz") or 2070.0
    fp32_peak = sm_count() * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    return {"kernel": "net_decompose_kernel", "samples_per_launch": samples, "outputs_per_launch": outs,
            "tensor": {"bound": "tensor", "flop": mma_flop, "achieved": mma_flop / t / 1e12, "peak": bf16,
                       "unit": "TFLOP/s", "frac": mma_flop / t / 1e12 / bf16,
                       "peak_note": "measured dense BF16, sustained (cuBLAS loop; the kernel runs inside a long step)"
                       if peaks.get("bf16_tflops_sustained") else "fallback 1700 TFLOP/s (sustained)"},
            "fp32": {"bound": "alu", "flop": fp32_flop, "achieved": fp32_flop / t / 1e12, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": fp32_flop / t / 1e12 / fp32_peak},
            "note": "bound in practice by the tcgen05 instruction pipe (~70 % busy, ncu), not by tensor math"}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def batched_main(args):
    """The batched form: 64 seeded volumes of uneven size, (s, D) per volume
    from the autotuner, all stages of all volumes in one CUDA graph."""
    import torch

    import phantom
    from paper_1708_07515_gb300 import autotune
    from paper_1708_07515_gb300.batch import BatchReconstructor, Instance
    torch.cuda.set_device(0)
    work = phantom.batched_workload()
    insts = [Instance(R, N, N, N, P) for N, P, R, _ in work]
    projs = [phantom.project_gpu(phantom.make_phantom(sd, N, 20), R, N, N, P) for N, P, R, sd in work]
    rates = autotune.measure_rates()
    br = BatchReconstructor(insts, rates=rates, persistent=args.persistent, tune_tiles=True)
    br.load(projs)
    br.capture()
    for _ in range(args.warmup):
        br.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        a.record(br.stream)
        for _ in range(args.steps):
            with torch.cuda.stream(br.stream):
                br.graph.replay()
        b.record(br.stream)
        torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    upd = sum(float(i.N) ** 3 * i.P for i in insts)
    out = {"metric": METRIC, "value": upd / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (projections generated on the GPU)",
           "config": {"workload": "batched_64_volumes_N64-384_P1.4N", "volumes": len(insts),
                      "step": "one CUDA-graph launch: bounds + filter + decompose + backproject of every volume",
                      "streams": len(br.lanes), "persistent_backprojection": br.batch is not None,
                      "tile_widths": br.tiles,
                      "choices": [[i.N, i.P, i.s, i.D] for i in insts], "rates": list(rates)},
           "gpu_launches": br.launches() * args.steps, "clocks": clk.summary()}
    print(json.dumps(out), flush=True)
    br.close()
    return 0


def slabs_main(args):
    """Slab-wise reconstruction (Sec. 2.2, piecemeal) through
    fdkod_reconstruct_slabs: a plan without the whole-volume workspace; each
    slab uploads only the detector rows it needs from page-locked host
    memory, filters, decomposes and backprojects them and copies the slab
    back, pipelined over three streams.  Timed on the host clock around whole
    reconstructions (the call is synchronous); device memory is compared with
    the whole-volume path."""
    import torch

    import paper_1708_07515_gb300 as fd
    import phantom
    torch.cuda.set_device(0)
    w = phantom.WORKLOADS[args.workload]
    ell = phantom.make_phantom(w.seed, w.N, w.n_ell)
    if w.N > 512:  # the CPU generator would take minutes
        proj = phantom.project_gpu(ell, w.R, w.Nu, w.Nv, w.P).cpu().numpy()
    else:
        proj = phantom.project(ell, w.R, w.Nu, w.Nv, w.P)
        if w.noise:
            phantom.add_noise(proj, w.noise, w.seed)
    proj = torch.from_numpy(proj).pin_memory()
    out = torch.empty((w.N, w.N, w.N), dtype=torch.float32).pin_memory()
    # whole-volume reference (and its device memory)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    base = torch.cuda.memory_allocated()
    with fd.Plan(w.R, w.N, w.Nu, w.Nv, w.P, w.s, w.D, qtype=args.qtype) as full:
        ref = full.backproject(full.filter(proj.cuda()))
        zs = [w.N // 3, 2 * w.N // 3]
        ref = ref[torch.as_tensor(zs, device="cuda")].cpu().numpy()
        torch.cuda.synchronize()
        full_bytes = torch.cuda.max_memory_allocated() - base + full.info["device_bytes"]
    torch.cuda.empty_cache()
    with fd.Plan(w.R, w.N, w.Nu, w.Nv, w.P, w.s, w.D, qtype=args.qtype, workspace=False) as plan:
        for _ in range(max(1, min(args.warmup, 2))):
            fd.reconstruct_slabs(plan, proj, args.slabs, out)
        torch.cuda.synchronize()
        steps = max(1, min(args.steps, 5))
        gc.collect()
        gc.disable()  # no collector pause of this Python harness inside the host-clocked calls
        with Clocks(0) as clk:
            t0 = time.perf_counter()
            for _ in range(steps):
                fd.reconstruct_slabs(plan, proj, args.slabs, out)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3 / steps
        gc.enable()
        slab_bytes = plan.info["device_bytes"] + plan.last_slab_device_bytes
        assert plan.device_status() == 0
        launches = 0
        for z0 in range(0, w.N, args.slabs):
            launches += 1 + (1 if w.D > 1 else 0) + 1  # filter rows, decompose band, backproject slab
    diff = float(np.abs(out.numpy()[zs] - ref).max() / np.abs(ref).max())
    print(json.dumps({
        "metric": METRIC, "value": float(w.N) ** 3 * w.P / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (host projections, host volume)",
        "config": {"workload": w.name, "slab_slices": args.slabs, "q_storage": args.qtype,
                   "step": "one slab-wise reconstruction: per slab, upload its detector rows, filter, decompose, "
                           "backproject, copy the slab back (three streams, double-buffered)",
                   "timer": "host clock (the call is synchronous)"},
        "device_bytes_peak": slab_bytes, "whole_volume_device_bytes_peak": full_bytes,
        "max_rel_diff_vs_whole_volume": diff, "gpu_launches": launches * steps, "clocks": clk.summary()}),
        flush=True)
    return 0


def split_main(args):
    """One volume split into z-slabs over the ranks (Sec. 2.2: a slab of
    slices reads only the detector rows the row formula b = z R / (R + x cos
    b + y sin b) allows).  Rank r reconstructs slab_partition(N, world)[r]
    from that band of rows alone (filter_rows + backproject_slab, the
    slab-wise entry points), with no exchange; the only collective is the max
    of the timings.  Strong scaling: the units are the whole volume's N^3 P
    effective updates, timed by the slowest rank."""
    import torch
    import torch.distributed as dist

    import paper_1708_07515_gb300 as fd
    import phantom
    from paper_1708_07515_gb300 import shard
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    w = phantom.WORKLOADS[args.workload]
    z0, z1 = shard.slab_partition(w.N, world)[rank]
    nz = z1 - z0
    # the same scan on every rank (same seeds); each keeps only its band of rows
    ell = phantom.make_phantom(w.seed, w.N, w.n_ell)
    plan = fd.Plan(w.R, w.N, w.Nu, w.Nv, w.P, w.s, w.D, qtype=args.qtype, workspace=False)
    v0, nrows = plan.slab_rows(z0, max(nz, 1))
    if w.noise and w.N <= 512:
        # the whole noisy scan (seeded), so the overlapping bands of two ranks agree
        full = phantom.make_projections(w)
        band = np.ascontiguousarray(full[:, v0:v0 + nrows])
        del full
    else:
        band = phantom.project(ell, w.R, w.Nu, w.Nv, w.P, rows=(v0, v0 + nrows))
    proj_d = torch.from_numpy(band).cuda()
    Qb = torch.empty(tuple(proj_d.shape), dtype=plan.q_torch_dtype, device="cuda")
    S_work = torch.empty(max(1, plan.slab_workspace_elems(nrows)), dtype=torch.float32, device="cuda")
    vol = torch.empty((max(nz, 1), w.N, w.N), dtype=torch.float32, device="cuda")

    def step():
        if nz > 0:
            plan.filter_rows(proj_d, v0, Qb)
            plan.backproject_slab(Qb, v0, S_work if w.D > 1 else None, z0, nz, vol)

    for _ in range(args.warmup):
        step()
    stream = torch.cuda.current_stream()
    with Clocks(local) as clk:
        barrier()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step()
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
    assert plan.device_status() == 0
    from paper_1708_07515_gb300.shard import max_over_ranks
    ms_step = max_over_ranks(t0.elapsed_time(t1)) / args.steps
    value = float(w.N) ** 3 * w.P / (ms_step * 1e-3)
    # end to end: the band up from page-locked host memory, the slab back
    band_h = torch.from_numpy(band).pin_memory()
    vol_h = torch.empty(tuple(vol.shape), dtype=torch.float32).pin_memory()

    def e2e_step():
        proj_d.copy_(band_h, non_blocking=True)
        step()
        vol_h.copy_(vol, non_blocking=True)

    for _ in range(2):
        e2e_step()
    barrier()
    torch.cuda.synchronize()
    a = time.perf_counter()
    n_e2e = max(2, min(args.steps, 10))
    for _ in range(n_e2e):
        e2e_step()
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks((time.perf_counter() - a) * 1e3) / n_e2e
    extra = {}
    if rank == 0 and nz > 0:
        import oracle
        oracle.build()
        zs = [z0, z0 + nz // 2, z1 - 1]
        Qo = np.zeros((w.P, w.Nv, w.Nu))
        Qo[:, v0:v0 + nrows] = oracle.filter_fft(band, w.R, v0=v0, Nv_det=w.Nv)
        ref = oracle.fdkod_slices(Qo, w.R, w.N, w.s, w.D, zs)
        got = vol[torch.as_tensor([z - z0 for z in zs], device="cuda")].cpu().numpy().astype(np.float64)
        extra["rel_rmse_vs_fp64_fdkod_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        extra["accuracy_slices"] = zs
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: seeded random-ellipsoid phantom, exact cone-beam projections"
                    + (f", {100 * w.noise:g}% Gaussian noise" if w.noise and w.N <= 512 else ""),
            "config": {**workload_config(w, args.qtype), "parallelism": f"one volume in {world} z-slabs",
                       "step": "per rank: filter its band of detector rows, decompose and backproject its slab",
                       "rank0_slab": [z0, z1], "rank0_rows": [v0, v0 + nrows]},
            "e2e": {"value": float(w.N) ** 3 * w.P / (ms_e2e * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": band.nbytes, "d2h_bytes_per_step": nz * w.N * w.N * 4,
                    "ms_per_step": ms_e2e, "note": "rank 0's band and slab; torch copies around the C ABI calls"},
            "gpu_launches": args.steps * (2 + (1 if w.D > 1 else 0)), "clocks": clk.summary(), **extra}),
            flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.batched:
        return batched_main(args)
    if args.slabs > 0:
        return slabs_main(args)
    if args.split == "z":
        return split_main(args)
    import torch
    import torch.distributed as dist

    import paper_1708_07515_gb300 as fd
    import phantom

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    w = phantom.WORKLOADS[args.workload]
    # each rank reconstructs its own scan (independent problems, weak scaling)
    ell = phantom.make_phantom(w.seed + rank, w.N, w.n_ell)
    gpu_inputs = w.N > 512  # the CPU generator would take minutes
    if gpu_inputs:
        proj_t = phantom.project_gpu(ell, w.R, w.Nu, w.Nv, w.P)
        if w.noise:
            gen = torch.Generator(device="cuda").manual_seed(w.seed + rank + 7919)
            sigma = w.noise * float(proj_t.max())
            for k in range(w.P):
                proj_t[k].add_(torch.randn(proj_t[k].shape, generator=gen, device="cuda"), alpha=sigma)
        proj = proj_t.cpu().numpy()
        del proj_t
    else:
        proj = phantom.project(ell, w.R, w.Nu, w.Nv, w.P)
        if w.noise:
            phantom.add_noise(proj, w.noise, w.seed + rank)

    taps = args.taps
    if taps == "learned":
        # 2D taps fitted on 4 noise-free training scans (other seeds), 16 slices each
        from paper_1708_07515_gb300 import learn
        train = [phantom.project_gpu(phantom.make_phantom(8000 + i, w.N, w.n_ell), w.R, w.Nu, w.Nv, w.P)
                 for i in range(4)]
        zs_fit = np.linspace(w.N // 8, w.N - 1 - w.N // 8, 16).round().astype(int)
        taps = learn.learn(w.R, w.N, w.P, w.s, w.D, 2, train, zs_fit)
        del train
    net_w = net_src = net_base = None
    if args.taps == "net":
        net_w, net_src, net_base = net_weights(args.net_weights, w.D)
        taps = "triangle" if net_base is None else net_base
    plan = fd.Plan(w.R, w.N, w.Nu, w.Nv, w.P, w.s, w.D, qtype=args.qtype, taps=taps)
    if net_w is not None:
        plan.set_net(net_w)
    info = plan.info
    stream = torch.cuda.current_stream()
    proj_d = torch.from_numpy(proj).cuda()
    Q = torch.empty((w.P, w.Nv, w.Nu), dtype=plan.q_torch_dtype, device="cuda")
    vol = torch.empty((w.N, w.N, w.N), dtype=torch.float32, device="cuda")
    upd_eff = float(w.N) ** 3 * w.P

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        plan.compute_bounds()
        if ev is not None:
            ev[1].record(stream)
        plan.filter(proj_d, Q)
        if ev is not None:
            ev[2].record(stream)
        plan.decompose_to_workspace(Q)  # the decomposed data stays in the plan's own workspace
        if ev is not None:
            ev[3].record(stream)
        plan.backproject_decomposed_workspace(vol)
        if ev is not None:
            ev[4].record(stream)

    launches_per_step = 4
    # --- device-resident timed region
    for _ in range(args.warmup):
        step()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    with Clocks(local) as clk:
        barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            step(evs[i])
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms_local = t0.elapsed_time(t1)
    stages = {name: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs)
              for i, name in enumerate(["bounds", "filter", "decompose", "backproject"])}
    assert plan.device_status() == 0, "staging window overflow"

    from paper_1708_07515_gb300.shard import max_over_ranks

    ms_total = max_over_ranks(ms_local)
    ms_step = ms_total / args.steps
    value = world * upd_eff / (ms_step * 1e-3)

    # --- plain FDK on the same GPU and data (filter + plain backprojection)
    def plain_step():
        plan.filter(proj_d, Q)
        plan.backproject_plain(Q, vol)

    for _ in range(max(1, args.warmup)):
        plain_step()
    n_plain = max(2, min(args.steps, 5))
    barrier()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(n_plain):
        plain_step()
    b.record(stream)
    torch.cuda.synchronize()
    ms_plain = max_over_ranks(a.elapsed_time(b)) / n_plain

    # --- end to end through the library's host-buffer call (fdkod_reconstruct):
    # every step uploads the scan's projections from page-locked host memory
    # and reads the whole volume back into it, inside the call (uploads in
    # bands of detector rows overlap the filter and the decomposition,
    # read-backs of groups of slices overlap the backprojection); the call is
    # synchronous, so the host clock times it
    if args.no_e2e:
        ms_e2e, n_e2e = None, 0
    else:
        proj_h = torch.from_numpy(proj).pin_memory()
        vol_h = torch.empty((w.N, w.N, w.N), dtype=torch.float32).pin_memory()
        for _ in range(max(2, min(args.warmup, 3))):
            fd.reconstruct(plan, proj_h, vol_h)
        n_e2e = max(2, min(args.steps, 30))
        barrier()
        torch.cuda.synchronize()
        t_calls = []
        gc.collect()
        gc.disable()  # no collector pause of this Python harness inside the host-clocked calls
        t_e0 = time.perf_counter()
        for _ in range(n_e2e):
            fd.reconstruct(plan, proj_h, vol_h)
            t_calls.append(time.perf_counter())
        gc.enable()
        ms_e2e = max_over_ranks((t_calls[-1] - t_e0) * 1e3) / n_e2e
        ms_calls = np.diff([t_e0] + t_calls) * 1e3
        del vol_h

    # --- accuracy at the measured configuration, against the FP64 oracle
    extra = {}
    cpu = None
    if rank == 0:
        import oracle
        oracle.build()
        vol_od = plan.backproject(Q).cpu().numpy()
        zs = [w.N // 2 - 1, w.N // 2]
        rows = rows_for_slices(w.N, w.Nv, w.R, zs)
        flat = np.array([k * w.Nv + v for k in range(w.P) for v in rows], dtype=np.int64)
        Qo = np.zeros((w.P, w.Nv, w.Nu))
        Qo.reshape(-1, w.Nu)[flat] = oracle.filter_rows(proj, w.R, flat)
        ref_fdk = oracle.fdk_slices(Qo, w.R, w.N, zs)
        if net_w is not None:
            # the net's oracle runs numpy per square: all squares up to 512^3,
            # 16 seeded squares beyond (their voxels only)
            nsq = 4 ** w.s
            squares = None if nsq <= 64 else sorted(np.random.default_rng(w.seed).choice(nsq, 16, replace=False))
            ref_od = oracle.fdkod_net_slices(Qo, w.R, w.N, w.s, w.D, plan.net, zs, act_round="bf16",
                                             squares=squares, taps=None if net_base is None else plan.taps)
        else:
            squares = None
            ref_od = oracle.fdkod_slices(Qo, w.R, w.N, w.s, w.D, zs,
                                         taps=None if args.taps == "triangle" else plan.taps)
        g = vol_od[zs].astype(np.float64)
        if squares is not None:
            mask = oracle.square_mask(w.N, w.s, squares)[None]
            g, ref_fdk = g * mask, ref_fdk * mask
            extra["accuracy_squares"] = [int(q) for q in squares]
        extra["rel_rmse_vs_fp64_fdkod_oracle"] = float(np.linalg.norm(g - ref_od) / np.linalg.norm(ref_od))
        extra["rel_rmse_vs_fp64_fdk_oracle"] = float(np.linalg.norm(g - ref_fdk) / np.linalg.norm(ref_fdk))
        extra["accuracy_slices"] = zs
        if not args.no_cpu_baseline:
            # seeded slices, one at a time, until about 10 s of oracle work
            order = np.random.default_rng(w.seed).permutation(w.N)
            done, t = [], 0.0
            while t < 10.0 and len(done) < min(64, w.N):
                z = int(order[len(done)])
                t += oracle_sample(w, proj, [z], oracle)
                done.append(z)
            cpu = {"value": len(done) * w.N * w.N * w.P / t, "unit": UNIT, "cores": oracle.max_threads(),
                   "kind": "oracle",
                   "sample": f"{len(done)} seeded slices of {w.name}, each: FP64 direct-convolution filter of "
                             f"the rows it needs + FP64 FDK-OD of the slice ({t:.1f} s total)"}
            # the oracle's plain FDK on the first of those slices, for the CPU-side speedup
            tf = oracle_sample_fdk(w, proj, done[:1], oracle)
            cpu["plain_fdk_value"] = w.N * w.N * w.P / tf
            cpu["plain_fdk_sample"] = f"slice {done[0]}: FP64 filter of its rows + FP64 plain FDK ({tf:.1f} s)"

    clocks = clk.summary()
    peaks = measured_peaks()
    bp_ms = stages["backproject"]
    upd_bp = float(w.N) ** 3 * (w.P // w.D)
    max_mhz = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    sms = sm_count(local)
    ops_peak = sms * FP32_LANES_PER_SM * max_mhz * 1e6 / 1e12
    ops_ach = OPS_PER_UPDATE * upd_bp / (bp_ms * 1e-3) / 1e12
    peak_tflops = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    achieved_tflops = FLOP_PER_UPDATE * upd_bp / (bp_ms * 1e-3) / 1e12
    smem_peak = sms * SMEM_BYTES_PER_CLK_PER_SM * max_mhz * 1e6 / 1e9
    smem_ach = SMEM_BYTES_PER_UPDATE * upd_bp / (bp_ms * 1e-3) / 1e9
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": ("synthetic: seeded random-ellipsoid phantom, exact cone-beam projections"
                     + (f", {100 * w.noise:g}% Gaussian noise" if w.noise else "")
                     + (" (projections generated on the GPU)" if gpu_inputs else "")),
            "config": {**workload_config(w, args.qtype, args.taps),
                       "step": "bounds + filter + decompose + backproject",
                       "l2": f"inputs larger than L2 (projections {proj.nbytes / 1e6:.0f} MB, decomposed data "
                             f"{info['decomposed_elems'] * 4 / 1e9:.2f} GB)",
                       "parallelism": f"{world} independent scans, one per GPU"},
            "e2e": None if ms_e2e is None else {
                "value": world * upd_eff / (ms_e2e * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": proj.nbytes, "d2h_bytes_per_step": w.N ** 3 * 4,
                "ms_per_step": ms_e2e, "steps": n_e2e,
                "ms_per_call_min_median_max": [round(float(f(ms_calls)), 3) for f in (np.min, np.median, np.max)],
                "slowest_call": int(np.argmax(ms_calls)),
                "value_at_median_call": world * upd_eff / (float(np.median(ms_calls)) * 1e-3),
                "call": "fdkod_reconstruct (C ABI, host buffers in and out, synchronous)",
                "python_gc": "disabled during the timed calls",
                "note": "host clock around whole calls; inside a call the upload (bands of detector rows) "
                        "overlaps the filter and the decomposition, the read-back (groups of slices) the "
                        "backprojection"},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": {"bound": "alu", "kernel": "FDK-OD backprojection",
                         "achieved": ops_ach, "peak": ops_peak, "unit": "TFLOP/s",
                         "frac": ops_ach / ops_peak,
                         "traffic": recorded_bp_traffic(args.workload if args.qtype == "f32" else ""),
                         "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                         "peak_note": f"{sms} SMs x 128 FP32 lanes x one operation per clock x {max_mhz:.0f} MHz "
                                      "(derived; an FMA counts one operation, as in the update's count)",
                         "per_launch_updates": upd_bp, "flop_per_update": OPS_PER_UPDATE,
                         "avg_launch_ms": bp_ms},
            "roofline_fma": {"achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                             "frac": achieved_tflops / peak_tflops, "flop_per_update": FLOP_PER_UPDATE,
                             "peak_note": f"{sms} SMs x 128 FP32 lanes x 2 (FMA) x {max_mhz:.0f} MHz"},
            "roofline_smem": {"achieved": smem_ach, "peak": smem_peak, "unit": "GB/s", "frac": smem_ach / smem_peak,
                              "bytes_per_update": SMEM_BYTES_PER_UPDATE},
            "roofline_stages": stage_rooflines(w, info, stages, args.qtype, peaks,
                                              plan.bounds()["T"] if w.D > 1 else None),
            **({"roofline_net": net_roofline(w, info, plan.bounds()["T"], stages, peaks), "net_weights": net_src,
                 "net_base": "triangle" if net_base is None else "learned linear taps (support 2D)"}
               if net_w is not None else {}),
            "stages_ms": stages,
            "plain_fdk": {"value": world * upd_eff / (ms_plain * 1e-3), "ms_per_step": ms_plain,
                          "step": "filter + plain backprojection"},
            "speedup_vs_plain_fdk": ms_plain / ms_step,
            "actual_updates_per_s": {"step": world * float(w.N) ** 3 * (w.P // w.D) / (ms_step * 1e-3),
                                     "backprojection": upd_bp / (bp_ms * 1e-3),
                                     "note": "N^3 P / D updates (the work FDK-OD does) per second"},
            "cpu_baseline": cpu,
            "clocks": clocks,
        }
        out.update(extra)
        print(json.dumps(out), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
