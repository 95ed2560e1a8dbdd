"""Pins of the two-belt (multirange) force in oracle/multirange.py (the
extension of Eq. SC_force that Sec. 2 names): exact isotropy of the E8 belt,
reduction to the single-belt force, zero net force, and the long-wave
expansion that gives both belts the same equation of state but different
third-order (surface-tension) terms.  CPU only."""

import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import lbm_oracle as o
from oracle import multirange as mr


def _double_factorial(n):
    return 1 if n <= 0 else n * _double_factorial(n - 2)


def _moment(vecs, weights, a, b, c):
    return sum(Fraction(wt) * int(v[0]) ** a * int(v[1]) ** b * int(v[2]) ** c for v, wt in zip(vecs, weights))


def _isotropic_to(vecs, weights, order):
    """True if every moment tensor of even order <= `order` is isotropic:
    <x^a y^b z^c> = e_2n (a-1)!! (b-1)!! (c-1)!! for a, b, c even, 0 else."""
    for two_n in range(2, order + 1, 2):
        e = _moment(vecs, weights, two_n, 0, 0) / _double_factorial(two_n - 1)
        for a in range(two_n + 1):
            for b in range(two_n + 1 - a):
                c = two_n - a - b
                m = _moment(vecs, weights, a, b, c)
                if a % 2 or b % 2 or c % 2:
                    want = 0
                else:
                    want = e * _double_factorial(a - 1) * _double_factorial(b - 1) * _double_factorial(c - 1)
                if m != want:
                    return False
    return True


def test_e8_belt_is_isotropic_to_eighth_order_and_d3q19_only_to_fourth():
    p = mr.e8_weights()
    vecs = mr.E8
    wts = [p[int((v * v).sum())] for v in vecs]
    assert len(vecs) == 92
    assert _moment(vecs, wts, 2, 0, 0) == 1
    assert all(w > 0 for w in p.values())
    assert _isotropic_to(vecs, wts, 8)
    # the test discriminates: the D3Q19 weights pass at 4th order, fail at 6th
    w19 = [Fraction(1, 18) if int((v * v).sum()) == 1 else Fraction(1, 36) for v in o.C]
    assert _isotropic_to(o.C, w19, 4)
    assert not _isotropic_to(o.C, w19, 6)


def test_two_belt_force_with_g2_zero_is_eq_sc_force():
    rho = 0.2 + 1.8 * np.random.default_rng(3).random((5, 6, 7))
    a, b = mr.two_belt_force(rho, -5.5, 0.0), o.shan_chen_force(rho, -5.5)
    assert np.abs(a - b).max() <= 4 * np.finfo(float).eps * np.abs(b).max()


def test_two_belt_force_has_no_net_momentum_on_a_periodic_box():
    rho = 0.2 + 1.8 * np.random.default_rng(4).random((9, 6, 7))
    F = mr.two_belt_force(rho, -3.0, -2.5)
    assert np.abs(F.sum(axis=(1, 2, 3))).max() <= 1e-13 * np.abs(F).sum()


@pytest.mark.parametrize("L", [64, 128])
def test_long_wave_expansion_same_eos_different_third_order(L):
    """For psi = sin(k x) each belt sum is cos(k x) (e2 k - e4x k^3 / 6 + O(k^5))
    with e2 = 1/3 for both belts (hence the common EoS P = rho cs2 + cs2 (G1 +
    G2) psi^2 / 2) and e4x = sum w c_x^4: 1/3 for D3Q19, larger for E8/3."""
    k = 2 * math.pi / L
    x = np.arange(L)
    psi = np.broadcast_to(np.sin(k * x)[None, None, :], (2, 2, L)).copy()
    p = mr.e8_weights()
    e4_19 = float(_moment(o.C, [Fraction(1, 18) if int((v * v).sum()) == 1 else Fraction(1, 36) for v in o.C], 4, 0, 0))
    e4_8 = float(_moment(mr.E8, [p[int((v * v).sum())] / 3 for v in mr.E8], 4, 0, 0))
    assert abs(e4_19 - 1 / 3) < 1e-15 and e4_8 > 1.5 * e4_19
    for vecs, wts, e4 in ((o.C, o.W, e4_19), (mr.E8, mr.P8 / 3.0, e4_8)):
        got = mr.belt_sum(psi, vecs, wts)[0, 0, 0]
        want = np.cos(k * x) * (k / 3.0 - e4 * k ** 3 / 6.0)
        assert np.abs(got - want).max() <= 0.1 * k ** 5 * 10, (L, np.abs(got - want).max())
        assert np.abs(mr.belt_sum(psi, vecs, wts)[1:]).max() < 1e-14
    # the O(k^3) difference between the belts is resolved
    d = mr.belt_sum(psi, mr.E8, mr.P8 / 3.0)[0, 0, 0] - mr.belt_sum(psi, o.C, o.W)[0, 0, 0]
    assert np.abs(d).max() > 0.5 * (e4_8 - e4_19) * k ** 3 / 6.0


def test_two_belt_sound_speed_follows_g1_plus_g2():
    """A standing density wave oscillates at c k with c^2 = cs2 (1 + (G1 + G2)
    psi psi'): the split G1 = -3, G2 = +1 sounds like the single belt at
    G = -2 (the bulk EoS depends on G1 + G2 only)."""
    from scipy.optimize import curve_fit

    L, rho0, steps = 128, 1.0, 700
    k = 2 * math.pi / L
    x = np.arange(L)
    p = o.Params(G=-3.0, tau=0.8, collision="srt")
    f = o.init_populations((rho0 + 1e-5 * np.cos(k * x))[None, None, :])
    amp = []
    for _ in range(steps):
        amp.append(2.0 / L * ((f.sum(0)[0, 0, :] - rho0) * np.cos(k * x)).sum())
        f = o.stream(mr.collide(f, p, 1.0))
    psi, dpsi = 1 - math.exp(-rho0), math.exp(-rho0)
    w0 = math.sqrt((1 + (-3.0 + 1.0) * psi * dpsi) / 3.0) * k

    def damped(t, A, w, g, ph):
        return A * np.cos(w * t + ph) * np.exp(-g * t)

    popt, _ = curve_fit(damped, np.arange(steps), np.array(amp), p0=[1e-5, w0, 1e-3, 0.0])
    assert abs(popt[1] / w0 - 1) < 2e-3, (popt[1], w0)
    w_g1_only = math.sqrt((1 - 3.0 * psi * dpsi) / 3.0) * k
    assert abs(popt[1] / w_g1_only - 1) > 0.1
