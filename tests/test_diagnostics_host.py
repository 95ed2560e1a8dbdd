"""Host-side diagnostics (neck radius, break-up time, growth-rate fit) on
synthetic inputs with known answers.  CPU only."""

import math

import numpy as np

from paper_1905_09554_gb300 import diagnostics as dg


def test_equivalent_and_neck_radius():
    R = np.array([3.0, 2.0, 5.0])
    area = math.pi * R ** 2
    assert np.allclose(dg.equivalent_radius(area), R)
    assert dg.neck_radius(area) == 2.0


def test_mode_amplitude_of_a_cosine_profile():
    nz = 64
    z = np.arange(nz)
    R = 8.0 * (1 + 0.05 * np.cos(2 * math.pi * z / nz))
    assert abs(dg.mode_amplitude(math.pi * R ** 2) - 0.4) < 1e-12


def test_breakup_time_interpolates_the_crossing():
    t = [0, 10, 20, 30]
    m = [2.0, 1.6, 1.0, 0.5]
    mid = 0.5 * (2.2 + 0.1)  # 1.15
    got = dg.breakup_time(t, m, 2.2, 0.1)
    assert abs(got - (10 + (1.6 - mid) / (1.6 - 1.0) * 10)) < 1e-12
    assert dg.breakup_time(t, [2, 2, 2, 2], 2.2, 0.1) is None
    assert dg.breakup_time(t, [0.5, 0.4, 0.3, 0.2], 2.2, 0.1) == 0.0


def test_growth_rate_recovers_an_exponential_and_stops_at_threshold():
    t = np.arange(0, 400, 10.0)
    a = 0.01 * np.exp(0.02 * t)
    a[t > 250] = 5.0  # beyond the stop amplitude: must be excluded
    assert abs(dg.growth_rate(t, a, t_start=50, a_stop=1.0) - 0.02) < 1e-12
    assert dg.growth_rate(t[:3], a[:3], t_start=0, a_stop=1.0) is None


def test_count_drops_counts_periodic_liquid_runs():
    rl, rv = 2.2, 0.1
    L, V = 2.0, 0.2  # liquid / vapour slice maxima
    assert dg.count_drops([L] * 8, rl, rv) == 1  # unbroken ligament
    assert dg.count_drops([V] * 8, rl, rv) == 0
    # two main drops and one satellite between them
    assert dg.count_drops([L, L, V, L, V, L, L, V], rl, rv) == 3
    # a run that wraps around z is one drop
    assert dg.count_drops([L, V, V, L, L, V, L, L], rl, rv) == 2
    # the mid density itself is not liquid
    assert dg.count_drops([1.15, V, L, V], rl, rv) == 1
