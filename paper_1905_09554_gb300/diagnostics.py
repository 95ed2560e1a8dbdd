"""Host-side ligament diagnostics built on lbm_diag's per-slice output
(Sec. 4 of the paper: minimum ligament radius, break-up time, perturbation
growth).  Pure numpy; no lattice arithmetic.

* equivalent radius R(z) = sqrt(A(z)/pi) from the liquid area A(z);
* neck radius min_z R(z);
* break-up: the first sample at which some slice holds no liquid, i.e.
  min_z max_xy rho < (rho_l + rho_v)/2, linearly interpolated between the
  two samples that bracket it;
* growth rate: least-squares slope of ln|a_k(t)|, a_k the cos(2 pi z / nz)
  coefficient of R(z, t), over a window [t_start, first t with
  |a_k| >= a_stop);
* drops after break-up: the maximal runs (periodic in z) of slices that hold
  liquid (max rho above the mid density); with the drops on the ligament's
  axis each run is one drop, and drops beyond the number of perturbation
  wavelengths are satellites (Fig. 2b's filled symbols);
* drops in 3D: the connected components (face neighbours, periodic in all
  three directions) of the cells with rho above the mid density, for a
  density field read back with lbm_moments; this also separates drops that
  sit side by side in a slice, which the per-slice count cannot.
"""

from __future__ import annotations

import math

import numpy as np


def equivalent_radius(area_z):
    return np.sqrt(np.asarray(area_z, dtype=float) / math.pi)


def neck_radius(area_z):
    return float(equivalent_radius(area_z).min())


def mode_amplitude(area_z, n_waves: int = 1):
    """cos(2 pi n z / nz) coefficient of R(z)."""
    R = equivalent_radius(area_z)
    nz = R.size
    return float(2.0 / nz * (R * np.cos(2.0 * math.pi * n_waves * np.arange(nz) / nz)).sum())


def breakup_time(times, min_maxrho, rho_l, rho_v):
    """Time at which min_z max_xy rho first falls below (rho_l + rho_v)/2,
    linearly interpolated between samples; None if it never does."""
    t = np.asarray(times, dtype=float)
    m = np.asarray(min_maxrho, dtype=float)
    mid = 0.5 * (rho_l + rho_v)
    below = np.nonzero(m < mid)[0]
    if below.size == 0:
        return None
    k = int(below[0])
    if k == 0:
        return float(t[0])
    t0, t1, m0, m1 = t[k - 1], t[k], m[k - 1], m[k]
    return float(t0 + (m0 - mid) / (m0 - m1) * (t1 - t0))


def growth_rate(times, amplitudes, t_start: float, a_stop: float, min_points: int = 4):
    """Slope of ln|a| over samples with t >= t_start taken before |a| first
    reaches a_stop; None if fewer than min_points samples qualify."""
    t = np.asarray(times, dtype=float)
    a = np.abs(np.asarray(amplitudes, dtype=float))
    hit = np.nonzero(a >= a_stop)[0]
    end = int(hit[0]) if hit.size else a.size
    sel = (np.arange(a.size) < end) & (t >= t_start) & (a > 0)
    if sel.sum() < min_points:
        return None
    return float(np.polyfit(t[sel], np.log(a[sel]), 1)[0])


def count_drops(maxrho_z, rho_l, rho_v):
    """Number of maximal periodic runs of z slices whose max rho exceeds
    (rho_l + rho_v)/2; 0 if no slice holds liquid, 1 if every slice does
    (an unbroken ligament)."""
    liquid = np.asarray(maxrho_z, dtype=float) > 0.5 * (rho_l + rho_v)
    if not liquid.any():
        return 0
    if liquid.all():
        return 1
    # a run starts where a liquid slice follows a dry one (wrapping around z)
    return int(np.count_nonzero(liquid & ~np.roll(liquid, 1)))


def drop_components(rho, rho_l, rho_v):
    """Connected components of the liquid (rho > (rho_l + rho_v)/2) of a
    periodic (nz, ny, nx) density field, cells joined across faces and across
    the periodic boundaries.  Returns the cell counts of the drops, largest
    first (an empty list if there is no liquid)."""
    from scipy import ndimage

    liquid = np.asarray(rho, dtype=float) > 0.5 * (rho_l + rho_v)
    lab, n = ndimage.label(liquid)  # face connectivity, not periodic
    if n == 0:
        return []
    parent = np.arange(n + 1)

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i

    for ax in range(3):
        lo = np.take(lab, 0, axis=ax).ravel()
        hi = np.take(lab, lab.shape[ax] - 1, axis=ax).ravel()
        both = (lo > 0) & (hi > 0)
        for i, j in set(zip(lo[both].tolist(), hi[both].tolist())):
            ri, rj = find(i), find(j)
            if ri != rj:
                parent[max(ri, rj)] = min(ri, rj)
    roots = np.array([find(i) for i in range(n + 1)])
    sizes = np.bincount(roots[lab[lab > 0]], minlength=n + 1)
    return sorted((int(v) for v in sizes if v > 0), reverse=True)
