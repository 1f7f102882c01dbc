"""Many reconstructions of uneven size in one CUDA graph.

Each volume gets its own plan (s and D chosen by the autotuner from the
Eq. 4-6 cost model with this GPU's measured rates), its own device buffers,
and the four stages of the hot path (bounds, filter, decomposition,
backprojection) for every volume are captured once into a single CUDA graph;
a batch then runs as one graph launch.  All kernels are libfdkod's; torch
only provides memory, streams and the graph object.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import autotune
from .fdkod import Plan


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
                 skip: int = 0):
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
        self.graph = None
        self.stream = torch.cuda.Stream()

    def _enqueue(self, stream_handle: int):
        for plan, p, Q, v in zip(self.plans, self.proj, self.Q, self.vol):
            plan.compute_bounds(stream_handle)
            plan.filter(p, Q, stream_handle)
            plan.backproject(Q, v, stream_handle)

    def run_eager(self):
        """All stages launched one by one on the current stream."""
        self._enqueue(int(self.torch.cuda.current_stream().cuda_stream))

    def capture(self):
        """Record the whole batch into one CUDA graph (after one eager run,
        which sets the kernels' shared-memory attributes outside capture)."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            self._enqueue(int(self.stream.cuda_stream))
        self.stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self._enqueue(int(self.stream.cuda_stream))
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
        for p in self.plans:
            p.close()
        self.plans = []
