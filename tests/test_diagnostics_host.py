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


def _flood_fill_sizes(liquid):
    """Component sizes by breadth-first search with periodic face neighbours."""
    nz, ny, nx = liquid.shape
    seen = np.zeros_like(liquid, dtype=bool)
    sizes = []
    for start in zip(*np.nonzero(liquid)):
        if seen[start]:
            continue
        seen[start] = True
        todo, n = [start], 0
        while todo:
            z, y, x = todo.pop()
            n += 1
            for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                c = ((z + dz) % nz, (y + dy) % ny, (x + dx) % nx)
                if liquid[c] and not seen[c]:
                    seen[c] = True
                    todo.append(c)
        sizes.append(n)
    return sorted(sizes, reverse=True)


def test_drop_components_in_3d():
    rl, rv = 2.0, 0.1
    z, y, x = np.indices((24, 16, 20))

    def ball(cz, cy, cx, r):
        return (z - cz) ** 2 + (y - cy) ** 2 + (x - cx) ** 2 <= r * r

    assert dg.drop_components(np.full((4, 4, 4), rv), rl, rv) == []
    one = np.where(ball(12, 8, 10, 4), rl, rv)
    assert dg.drop_components(one, rl, rv) == [int(ball(12, 8, 10, 4).sum())]
    # a drop centred on the corner wraps across all three periodic faces
    wrap = ball(0, 0, 0, 3) | ball(24, 0, 0, 3) | ball(0, 16, 0, 3) | ball(0, 0, 20, 3) | \
        ball(24, 16, 0, 3) | ball(24, 0, 20, 3) | ball(0, 16, 20, 3) | ball(24, 16, 20, 3)
    assert len(dg.drop_components(np.where(wrap, rl, rv), rl, rv)) == 1
    # two drops side by side in the same slices: the per-slice count sees one
    pair = ball(12, 8, 4, 3) | ball(12, 8, 15, 3)
    rho = np.where(pair, rl, rv)
    assert len(dg.drop_components(rho, rl, rv)) == 2
    assert dg.count_drops(rho.max(axis=(1, 2)), rl, rv) == 1
    # an unbroken ligament along z (closed through the periodic boundary)
    lig = (y - 8) ** 2 + (x - 10) ** 2 <= 9
    assert dg.drop_components(np.where(lig, rl, rv), rl, rv) == [int(lig.sum())]
    # brute force on random sparse fields
    rng = np.random.default_rng(11)
    for frac in (0.15, 0.3, 0.45):
        liq = rng.random((7, 6, 5)) < frac
        assert dg.drop_components(np.where(liq, rl, rv), rl, rv) == _flood_fill_sizes(liq)
