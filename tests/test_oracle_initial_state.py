"""Pins of the oracle's ligament initial state (Sec. 3, "Simulations set-up")
against what the set-up fixes, without restating its formula:

* a node that lies exactly on the perturbed surface holds the mid density
  (rho_l + rho_v)/2, on an odd box (axis through a node) and an even box
  (axis between four nodes), at the crest, trough and node of the cosine;
* far inside and far outside the density tends to rho_l and rho_v with the
  exponential tail of a tanh edge;
* the radial slope at the surface is -(rho_l - rho_v) / (2 W);
* the liquid area of every slice equals the Sommerfeld integral of a disc
  with a tanh edge, pi R(z)^2 + pi^3 W^2 / 12 (exact for the quadratic
  area function; the lattice sum equals the integral to ~1e-9 for W = 2).

A dropped factor 1/2, a width read as 2W, a sine for the cosine, a wrong
number of wavelengths or an off-centre axis each fails one of them.
"""

import math

import numpy as np
import pytest

from oracle import initial_state as ini

RL, RV = 2.3, 0.1
MID = 0.5 * (RL + RV)


@pytest.mark.parametrize("z,nodes", [
    # odd 21 x 21 box, axis through node (10, 10); R0 = 5, eps = 0.2, nz = 8:
    # R(0) = 6, R(2) = 5, R(4) = 4 (crest, node and trough of the cosine)
    (0, [(16, 10), (4, 10), (10, 16), (10, 4)]),
    (2, [(15, 10), (5, 10), (13, 14), (7, 6), (10, 15)]),
    (4, [(14, 10), (6, 10), (10, 14), (10, 6)]),
])
def test_mid_density_on_surface_nodes_odd_box(z, nodes):
    rho = ini.ligament_density(21, 21, 8, 5.0, 0.2, RL, RV)
    for x, y in nodes:
        assert abs(rho[z, y, x] - MID) <= 1e-14, (z, x, y)
    # the axis node is the most liquid one of its slice
    assert rho[z, 10, 10] == rho[z].max()


def test_mid_density_on_surface_nodes_even_box():
    """20 x 20 box: the axis is at (9.5, 9.5), so the eight nodes at offsets
    (+-3.5, +-0.5) and (+-0.5, +-3.5) lie at r = sqrt(12.5)."""
    R = math.sqrt(12.5)
    rho = ini.ligament_density(20, 20, 3, R, 0.0, RL, RV)
    for x, y in [(13, 9), (13, 10), (6, 9), (6, 10), (9, 13), (10, 13), (9, 6), (10, 6)]:
        for z in range(3):
            assert abs(rho[z, y, x] - MID) <= 1e-14, (x, y)
    # the four central nodes are equally liquid (axis between them)
    c = rho[0, 9:11, 9:11]
    assert np.ptp(c) <= 1e-15


def test_bulk_limits_follow_the_tanh_tail():
    """Inside: rho_l - rho(axis) = D e^{-2R/W} / (1 + e^{-2R/W}); outside at
    distance d beyond the surface: rho - rho_v = D / (1 + e^{2d/W})."""
    W, R0, n = 2.0, 9.0, 41
    rho = ini.ligament_density(n, n, 4, R0, 0.0, RL, RV, width=W)
    D = RL - RV
    e = math.exp(-2.0 * R0 / W)
    assert 0.0 < RL - rho[0, 20, 20] <= D * e * (1 + 1e-12)
    d = math.hypot(20, 20) - R0  # corner node
    assert 0.0 < rho[0, 0, 0] - RV <= D * math.exp(-2.0 * d / W) * (1 + 1e-12)
    assert rho[0, 20, 20] > rho[0, 20, 35] > rho[0, 0, 0]


def test_slope_at_the_surface_is_half_the_contrast_over_the_width():
    """Move the surface across a fixed node (eps = 0, R0 = 5 -/+ h) and
    difference: d rho / dR at r = R equals (rho_l - rho_v) / (2 W)."""
    for W in (1.0, 2.0, 3.0):
        h = 1e-5
        lo = ini.ligament_density(21, 21, 1, 5.0 - h, 0.0, RL, RV, width=W)[0, 10, 15]
        hi = ini.ligament_density(21, 21, 1, 5.0 + h, 0.0, RL, RV, width=W)[0, 10, 15]
        slope = (hi - lo) / (2 * h)
        assert abs(slope - (RL - RV) / (2 * W)) <= 1e-8, W


@pytest.mark.parametrize("R0,eps,n_waves,width", [(16.0, 0.08, 1, 2.0), (16.0, -0.1, 2, 2.0), (18.0, 0.05, 3, 2.2)])
def test_slice_area_equals_the_sommerfeld_integral(R0, eps, n_waves, width):
    """A(z) = sum_xy (rho - rho_v)/(rho_l - rho_v) against
    int_0^inf 2 pi r dr / (1 + e^{2(r - R)/W}) = pi R^2 + (pi^2/6)(W/2)^2 2 pi,
    R = R0 (1 + eps cos(2 pi n z / nz))."""
    n, nz = 84, 36
    rho = ini.ligament_density(n, n, nz, R0, eps, RL, RV, width=width, n_waves=n_waves)
    A = ((rho - RV) / (RL - RV)).sum(axis=(1, 2))
    z = np.arange(nz)
    R = R0 * (1.0 + eps * np.cos(2.0 * math.pi * n_waves * z / nz))
    want = math.pi * R ** 2 + math.pi ** 3 * width ** 2 / 12.0
    assert np.abs(A / want - 1.0).max() <= 1e-7
    # the perturbation is a cosine: the crest is at z = 0
    assert np.argmax(A) == 0 if eps > 0 else np.argmin(A) == 0


def test_surface_radius_at_crest_trough_and_node():
    assert ini.surface_radius(0, 40, 10.0, 0.1) == pytest.approx(11.0, abs=1e-14)
    assert ini.surface_radius(20, 40, 10.0, 0.1) == pytest.approx(9.0, abs=1e-14)
    assert ini.surface_radius(10, 40, 10.0, 0.1) == pytest.approx(10.0, abs=1e-14)
    assert ini.surface_radius(10, 40, 10.0, 0.1, n_waves=2) == pytest.approx(9.0, abs=1e-14)
