"""Choice of the decomposition level s and decimation factor D.

The paper's cost model (Sec. 2.2, Eq. 4-6): reconstruction costs
C1 N^4 / 2^s and decomposition C2 N^3 2^s, so the total is smallest at
2^s = sqrt(C1 N / C2).  Here the two constants come from this GPU: the
backprojection's voxel-update rate and the decomposition's shifted-sample
rate, each measured on one small probe plan, give
    t_rec(s, D) = N^3 (P / D) / rate_bp
    t_dec(s)    = sum_q P Nv T_q / rate_dec ~ kappa 2^s N Nv P / rate_dec,
and a short measured search around the model's optimum picks the plan.
choose_tile then picks the backprojection's tile shape -- the width of the
staging window each 16 x 16 x 32-voxel tile reads per view (fdkod_set_tile)
-- by timing the plan's own backprojection with each valid width.
D is kept a divisor of P and at most 2^s (one decimation stage per
decomposition stage, Sec. 2.2); `skip` lowers it by that many stages for
quality (the paper skips one stage in its measurements, Sec. 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass


@dataclass
class Choice:
    s: int
    D: int
    predicted_ms: float
    measured_ms: float | None = None


def divisors_up_to(P: int, limit: int) -> list[int]:
    return [d for d in range(1, max(1, limit) + 1) if P % d == 0]


def decimation_for(P: int, s: int, skip: int = 0) -> int:
    """Largest divisor of P not above 2^(s - skip)."""
    cap = 2 ** max(0, s - skip)
    return max(divisors_up_to(P, cap))


def model_ms(N: int, P: int, s: int, D: int, rate_bp: float, rate_dec: float, kappa: float = 1.45) -> float:
    """Eq. 4-6 with measured rates (updates/s, samples/s)."""
    t_rec = float(N) ** 3 * (P / D) / rate_bp
    t_dec = 0.0 if D == 1 else kappa * (2 ** s) * float(N) * N * P / rate_dec
    return 1e3 * (t_rec + t_dec)


def optimal_s_model(N: int, rate_bp: float, rate_dec: float, kappa: float = 1.45) -> float:
    """Continuous optimum of Eq. 6 with D = 2^s: 2^s = sqrt(N rate_dec / (kappa rate_bp))."""
    return 0.5 * math.log2(max(1.0, N * rate_dec / (kappa * rate_bp)))


def measure_rates(N: int = 128, P: int = 120) -> tuple[float, float]:
    """Backprojection updates/s and decomposition samples/s of this GPU on a
    small probe scan (random filtered data; timing only)."""
    import torch

    from .fdkod import Plan
    plan = Plan(4.0 * N, N, N, N, P, 2, 4)
    try:
        Q = torch.randn((P, N, N), device="cuda")
        S = plan.decompose(Q)
        vol = torch.empty((N, N, N), device="cuda")

        def t(fn, reps=3):
            fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps * 1e-3

        t_bp = t(lambda: plan.backproject_decomposed(S, vol))
        t_dec = t(lambda: plan.decompose(Q, S))
        T = plan.bounds()["T"]
        samples = float(P) * N * float(T.sum())
        return float(N) ** 3 * (P // 4) / t_bp, samples / t_dec
    finally:
        plan.close()


def choose(N: int, P: int, rate_bp: float, rate_dec: float, skip: int = 0, smax: int = 7,
           timer=None, search: int = 1) -> Choice:
    """Pick (s, D): the model's best s, then (if a timer is given) measure
    s-search..s+search and keep the fastest.  timer(s, D) -> milliseconds."""
    smax = min(smax, int(math.floor(math.log2(max(1, N)))))
    cands = []
    for s in range(0, smax + 1):
        D = decimation_for(P, s, skip)
        cands.append(Choice(s, D, model_ms(N, P, s, D, rate_bp, rate_dec)))
    best = min(cands, key=lambda c: c.predicted_ms)
    if timer is None:
        return best
    tried = []
    for c in cands:
        if abs(c.s - best.s) <= search:
            c.measured_ms = float(timer(c.s, c.D))
            tried.append(c)
    return min(tried, key=lambda c: c.measured_ms)


TILE_WIDTHS = (32, 48, 64, 96, 128)


def tile_candidates(min_cols: int, count: int = 3) -> list[int]:
    """The narrowest valid staging-window width and the next wider ones."""
    return [w for w in TILE_WIDTHS if w >= min_cols][:count] if min_cols > 0 else []


def choose_tile(plan, reps: int = 3, count: int = 3) -> tuple[int, dict]:
    """Time the plan's FDK-OD backprojection (from its decomposed workspace,
    or from Q when D = 1) with each candidate window width, keep the fastest
    (set on the plan) and return (width, {width: ms}).  Data values do not
    change the timing, so zero inputs serve."""
    import torch
    _, narrowest = plan.tile
    cands = tile_candidates(narrowest, count)
    if len(cands) < 2:
        return plan.tile[0], {}
    Q = torch.zeros((plan.P, plan.Nv, plan.Nu), dtype=plan.q_torch_dtype, device="cuda")
    vol = torch.empty((plan.N, plan.N, plan.N), dtype=torch.float32, device="cuda")
    if plan.D > 1:
        plan.decompose_to_workspace(Q)
    times = {}
    for w in cands:
        plan.set_tile(w)
        run = (lambda: plan.backproject(Q, vol)) if plan.D == 1 else \
            (lambda: plan.backproject_decomposed_workspace(vol))
        run()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            run()
        b.record()
        torch.cuda.synchronize()
        times[w] = a.elapsed_time(b) / reps
    best = min(times, key=times.get)
    plan.set_tile(best)
    return best, times
