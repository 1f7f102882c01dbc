"""Many reconstructions of uneven size in one CUDA graph.

Each volume gets its own plan (s and D chosen by the autotuner from the
Eq. 4-6 cost model with this GPU's measured rates) and its own device
buffers.  The bounds, filter and decomposition of every volume are spread
over several streams (largest estimated cost first, each to the
least-loaded stream; in the graph they become parallel branches), each
followed on its stream by the volume's backprojection, so one volume's
filter and decomposition overlap other volumes' backprojections.  With
persistent=True the backprojections of all volumes -- most of the work --
are instead one persistent launch after every decomposition
(fdkod_batch_backproject: a work list of (volume, tile, z-slab) items,
largest volumes first, taken by as many CTAs as the GPU holds); it gives
the same volumes bit for bit but gives up that overlap (a kernel cannot
wait for another launch's results), which costs more than it saves (207
against 187 ms for 64 volumes of N 64-384).  The whole batch is captured
once into a single CUDA graph and runs as one graph launch.  All kernels
are libfdkod's; torch only provides memory, streams and the graph object.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import autotune
from .fdkod import BatchBackprojection, FdkodError, Plan


def work_estimate(inst) -> float:
    """Relative cost of one volume: its backprojection updates N^3 P / D."""
    return float(inst.N) ** 3 * inst.P / max(1, inst.D)


def assign_lanes(costs: list[float], lanes: int) -> list[int]:
    """Longest-processing-time-first: each volume, largest first, goes to the
    lane with the least work so far.  Returns the lane of every volume."""
    load = [0.0] * lanes
    out = [0] * len(costs)
    for k in sorted(range(len(costs)), key=lambda i: -costs[i]):
        j = min(range(lanes), key=lambda i: load[i])
        out[k] = j
        load[j] += costs[k]
    return out


@dataclass
class Instance:
    R: float
    N: int
    Nu: int
    Nv: int
    P: int
    s: int = -1  # chosen by the autotuner when < 0
    D: int = -1


class BatchReconstructor:
    def __init__(self, instances: list[Instance], qtype: str = "f32", rates: tuple[float, float] | None = None,
                 skip: int = 0, streams: int = 4, persistent: bool = False, tune_tiles: bool = False):
        import torch
        self.torch = torch
        self.instances = instances
        if any(i.s < 0 or i.D < 0 for i in instances) and rates is None:
            rates = autotune.measure_rates()
        self.rates = rates
        self.plans, self.proj, self.Q, self.vol = [], [], [], []
        for inst in instances:
            if inst.s < 0 or inst.D < 0:
                c = autotune.choose(inst.N, inst.P, rates[0], rates[1], skip=skip)
                inst.s, inst.D = c.s, c.D
            plan = Plan(inst.R, inst.N, inst.Nu, inst.Nv, inst.P, inst.s, inst.D, qtype=qtype)
            self.plans.append(plan)
            self.proj.append(torch.empty((inst.P, inst.Nv, inst.Nu), dtype=torch.float32, device="cuda"))
            self.Q.append(torch.empty((inst.P, inst.Nv, inst.Nu), dtype=plan.q_torch_dtype, device="cuda"))
            self.vol.append(torch.empty((inst.N, inst.N, inst.N), dtype=torch.float32, device="cuda"))
        # tile shape per volume (the backprojection's staging-window width),
        # timed on the volume's own plan
        self.tiles = [autotune.choose_tile(p)[0] if tune_tiles else p.tile[0] for p in self.plans]
        self.graph = None
        self.stream = torch.cuda.Stream()
        self.lanes = [torch.cuda.Stream() for _ in range(max(1, streams))]
        self.assign = assign_lanes([work_estimate(i) for i in instances], len(self.lanes))
        self.batch = None
        if persistent:
            try:
                self.batch = BatchBackprojection(self.plans, [Q if i.D == 1 else None for i, Q in
                                                              zip(instances, self.Q)], self.vol)
            except FdkodError as e:
                if e.status != -2:
                    raise

    def launches(self) -> int:
        """Kernel launches per batch: bounds, filter and the decomposition
        (only when D > 1) of every volume, plus one persistent
        backprojection (or one backprojection per volume)."""
        per = sum(3 if i.D > 1 else 2 for i in self.instances)
        return per + (1 if self.batch is not None else len(self.instances))

    def _enqueue(self, main):
        """Every volume's stages on its lane; the lanes fork from and join
        back into `main` (in a capture they become parallel graph branches)."""
        for lane in self.lanes:
            lane.wait_stream(main)
        for k, (inst, plan, p, Q, v) in enumerate(zip(self.instances, self.plans, self.proj, self.Q, self.vol)):
            h = int(self.lanes[self.assign[k]].cuda_stream)
            plan.compute_bounds(h)
            plan.filter(p, Q, h)
            if self.batch is None:
                plan.backproject(Q, v, h)
            elif inst.D > 1:
                plan.decompose_to_workspace(Q, h)
        for lane in self.lanes:
            main.wait_stream(lane)
        if self.batch is not None:
            self.batch.run(int(main.cuda_stream))

    def run_eager(self):
        """All stages launched one by one (forked over the lanes from the
        current stream and joined back into it)."""
        self._enqueue(self.torch.cuda.current_stream())

    def capture(self):
        """Record the whole batch into one CUDA graph (after one eager run,
        which sets the kernels' shared-memory attributes outside capture)."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            self._enqueue(self.stream)
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self._enqueue(self.stream)
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def load(self, projections):
        """Copy host or device projections into the batch's input buffers."""
        for dst, src in zip(self.proj, projections):
            dst.copy_(self.torch.as_tensor(src), non_blocking=True)

    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        for p in self.plans:
            p.close()
        self.plans = []
