"""Host logic of the (s, D) choice: Eq. 4-6 cost model and the constraints
on D (a divisor of P, at most 2^(s - skip))."""
import math

import pytest

from paper_1708_07515_gb300 import autotune


def test_decimation_is_a_divisor_of_P_within_the_stage_cap():
    assert autotune.decimation_for(720, 3) == 8
    assert autotune.decimation_for(720, 3, skip=1) == 4
    assert autotune.decimation_for(179, 4) == 1          # prime view count: crop only
    assert autotune.decimation_for(358, 5) == 2
    for P in (90, 134, 179, 269, 358, 538, 720):
        for s in range(0, 6):
            D = autotune.decimation_for(P, s)
            assert P % D == 0 and D <= 2 ** s


def test_model_optimum_matches_the_closed_form():
    """Eq. 6 with D = 2^s: N^4/2^s * a + N^3 2^s * b is smallest where
    2^s = sqrt(a N / b); the discrete choice sits next to it."""
    N, P = 512, 720 * 16  # P divisible by every 2^s considered
    rate_bp, rate_dec = 1.5e12, 4e11
    s_star = autotune.optimal_s_model(N, rate_bp, rate_dec)
    best = autotune.choose(N, P, rate_bp, rate_dec)
    assert abs(best.s - s_star) <= 1.0
    costs = [autotune.model_ms(N, P, s, 2 ** s, rate_bp, rate_dec) for s in range(8)]
    assert costs.index(min(costs)) == best.s


def test_faster_decomposition_moves_the_optimum_up():
    a = autotune.choose(1024, 720 * 64, 1.5e12, 1e11)
    b = autotune.choose(1024, 720 * 64, 1.5e12, 1e13)
    assert b.s >= a.s


def test_measured_search_keeps_the_fastest():
    calls = []

    def timer(s, D):
        calls.append((s, D))
        return 10.0 + (s - 2) ** 2

    c = autotune.choose(256, 360, 1.5e12, 4e11, timer=timer)
    assert c.measured_ms == min(10.0 + (s - 2) ** 2 for s, _ in calls)
    assert len(calls) <= 3


def test_lane_assignment_balances_longest_first():
    from paper_1708_07515_gb300.batch import assign_lanes
    costs = [5.0, 1.0, 4.0, 3.0, 3.0, 2.0]
    lanes = assign_lanes(costs, 2)
    assert lanes == [0, 0, 1, 1, 0, 1]
    load = [sum(c for c, l in zip(costs, lanes) if l == j) for j in range(2)]
    assert max(load) - min(load) <= max(costs)
    # one lane: everything on it; more lanes than volumes: one volume each
    assert assign_lanes(costs, 1) == [0] * 6
    assert sorted(assign_lanes(costs[:3], 5)) == [0, 1, 2]


def test_tile_candidates():
    from paper_1708_07515_gb300 import autotune
    assert autotune.tile_candidates(48) == [48, 64, 96]
    assert autotune.tile_candidates(96, count=5) == [96, 128]
    assert autotune.tile_candidates(128) == [128]
    assert autotune.tile_candidates(0) == []
