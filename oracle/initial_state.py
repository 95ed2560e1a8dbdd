"""Initial state of the ligament break-up problem (Sec. 3, "Simulations
set-up"), in plain FP64, for checking the library's device-side set-up.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may import this module; the library never does.  It
shares no code with the CUDA sources or with the seeded input generators.

Sec. 3 starts the instability from a liquid cylinder whose radius carries a
sinusoidal perturbation of amplitude delta along the cylinder axis.  The
reading used here (and by the library's ``lbm_init_ligament``):

* the cylinder axis is the z axis of the box and passes through the centre of
  the cross-section, ((nx - 1)/2, (ny - 1)/2) in cell-node coordinates, so an
  odd box has a node on the axis and an even box has the axis between four
  nodes;
* the surface radius is R(z) = R0 (1 + eps cos(2 pi n z / nz)), i.e.
  delta = eps R0, with n whole wavelengths in the periodic box (the paper
  writes a sine of 4 pi x / L_x: two wavelengths; a cosine only moves the
  origin along the axis);
* across the surface the density goes from rho_l inside to rho_v outside
  along a tanh profile whose length scale is the interface width W:
  rho(r, z) = rho_v + (rho_l - rho_v) (1 - tanh((r - R(z)) / W)) / 2,
  with r the distance of the cell node from the axis;
* the fluid starts at rest.

Parity unpinned: none.  ``tests/test_oracle_initial_state.py`` checks this
module against what the set-up fixes without restating its formula (the
mid density on nodes that lie on the surface of odd and even boxes, the bulk
limits, the slope at the surface, and the liquid area of each slice against
the exact Sommerfeld integral pi R(z)^2 + pi^3 W^2 / 12 of a tanh-edged disc).
"""

from __future__ import annotations

import math

import numpy as np


def surface_radius(z, nz, R0, eps, n_waves=1):
    """R(z) = R0 (1 + eps cos(2 pi n z / nz)) for the plane index z."""
    return R0 * (1.0 + eps * math.cos(2.0 * math.pi * n_waves * z / nz))


def ligament_density(nx, ny, nz, R0, eps, rho_l, rho_v, width=2.0, n_waves=1):
    """Density field (nz, ny, nx), x fastest, of the perturbed ligament at
    t = 0.  Built slice by slice: for each plane z the surface radius R(z),
    then every node's distance from the axis and its tanh-profile density."""
    xc = 0.5 * (nx - 1)
    yc = 0.5 * (ny - 1)
    # distance of every node of a cross-section from the axis (same for all z)
    dx = np.arange(nx, dtype=np.float64) - xc
    dy = np.arange(ny, dtype=np.float64) - yc
    r = np.hypot(dy[:, None], dx[None, :])
    rho = np.empty((nz, ny, nx), dtype=np.float64)
    for z in range(nz):
        Rz = surface_radius(z, nz, R0, eps, n_waves)
        liquid_fraction = 0.5 * (1.0 - np.tanh((r - Rz) / width))
        rho[z] = rho_v + (rho_l - rho_v) * liquid_fraction
    return rho

