"""Surface tension, coexistence densities and the viscosity calibration of
the break-up runs (Sec. 3), measured with the GPU step.

Sec. 3 fixes G0 = -5.3 and Oh = 0.1 and, for every ligament radius R0,
chooses the relaxation time so that Oh = mu / sqrt(rho_l sigma R0) with
mu = rho_l nu, nu = cs2 (tau - 1/2) (Eq. Oh_Tcap).  With SRT the surface
tension and the coexistence densities depend on tau, so the paper iterates:
Laplace test (three static droplets) -> sigma -> the tau that meets Oh ->
Laplace test again, until two consecutive sigma agree (it stops at 5%); flat
interfaces then give rho_l and rho_v.  With MRT sigma does not depend on
tau and one pass suffices.  This module implements those steps:

* `pressure`: the equation of state of the method, P = cs2 rho + cs2 G psi^2 / 2
  (Eq. EOS_SC), psi = rho0 (1 - exp(-rho / rho0));
* `flat_coexistence`: a slab of liquid in a periodic box run to steady
  state; rho_l, rho_v are the densities in the middle of each phase;
* `laplace_sigma`: static spherical droplets of three radii (16, 20, 24 in
  boxes of 4 R); the pressure jump between the droplet centre and the far
  vapour against 1/R (R the equimolar radius), dp = 2 sigma / R;
* `tau_for_oh`: the relaxation time that gives Oh for sigma, rho_l, R0;
* `calibrate_tau`: the fixed-point iteration tau -> (sigma, rho_l) -> tau.

All lattice work runs through `lbm.Lattice` (the CUDA library); this file
holds only the host-side set-up, the fits and the iteration.
"""

from __future__ import annotations

import math

import numpy as np

CS2 = 1.0 / 3.0


def pressure(rho, G, rho0=1.0, G2=0.0):
    """Bulk pressure of the Shan-Chen fluid, Eq. EOS_SC; with the two-belt
    force the interaction strength is G + G2."""
    rho = np.asarray(rho, dtype=float)
    psi = rho0 * (1.0 - np.exp(-rho / rho0))
    return CS2 * rho + 0.5 * CS2 * (G + G2) * psi ** 2


def tau_for_oh(Oh, sigma, rho_l, R0):
    """tau with Oh = rho_l nu / sqrt(rho_l sigma R0), nu = cs2 (tau - 1/2)
    (Eq. Oh_Tcap)."""
    nu = Oh * math.sqrt(sigma * R0 / rho_l)
    return 0.5 + nu / CS2


def t_cap(sigma, rho_l, R0):
    """Capillary time sqrt(rho_l R0^3 / sigma), Eq. Oh_Tcap."""
    return math.sqrt(rho_l * R0 ** 3 / sigma)


def _run_to_steady(L, max_steps, check_every, tol):
    """Step until the density field changes by less than tol (max abs) over
    check_every steps, or max_steps; returns (rho, steps)."""
    rho_prev = L.moments()[0]
    steps = 0
    while steps < max_steps:
        L.step(check_every)
        steps += check_every
        rho = L.moments()[0]
        if np.abs(rho - rho_prev).max() < tol:
            return rho, steps
        rho_prev = rho
    return rho_prev, steps


def _lattice(shape, G, tau, collision, rates, storage, G2=0.0):
    from . import lbm
    nx, ny, nz = shape
    return lbm.Lattice(nx, ny, nz, G=G, tau=tau, collision=collision, rates=rates, storage=storage, G2=G2)


def flat_coexistence(G, tau, collision="srt", rates=None, storage="f64", length=64, width=2.0,
                     rho_guess=(2.1, 0.1), max_steps=40000, check_every=500, tol=1e-10, G2=0.0):
    """Coexistence densities from a flat liquid slab (normal along z) in a
    4 x 4 x length periodic box: (rho_l, rho_v, steps)."""
    rl, rv = rho_guess
    z = np.arange(length)
    d = np.abs(z - (length - 1) / 2.0) - length / 4.0  # < 0 inside the slab
    prof = rv + 0.5 * (rl - rv) * (1.0 - np.tanh(d / width))
    rho0 = np.broadcast_to(prof[:, None, None], (length, 4, 4)).copy()
    with _lattice((4, 4, length), G, tau, collision, rates, storage, G2) as L:
        L.set_density(rho0)
        rho, steps = _run_to_steady(L, max_steps, check_every, tol)
    col = rho[:, 0, 0]
    return float(col[length // 2]), float(col[0]), steps


def laplace_sigma(G, tau, collision="srt", rates=None, storage="f64", radii=(16.0, 20.0, 24.0),
                  box_factor=4.0, width=2.0, rho_guess=(2.1, 0.1), max_steps=30000, check_every=1000,
                  tol=1e-9, G2=0.0):
    """Surface tension from the Laplace test on static droplets.

    Each droplet of initial radius R sits in a periodic box of about
    box_factor * R cells a side.  The vapour around a droplet of this model
    is denser than at a flat interface (by ~10% at R = 20) and takes its mass
    from the droplet, so the vapour volume is kept a modest multiple of the
    droplet's: in a box of 80 cells a droplet started at R = 12 shrinks to
    R = 8.8.  Measured: rho_in (mean of the 4^3 centre cells), rho_out (the
    corner cell), the equimolar radius from the total mass, and
    dp = P(rho_in) - P(rho_out); sigma from the Laplace law dp = 2 sigma / R
    by least squares through the origin.  The free line dp = a + 2 s / R is
    also fitted (s = `sigma_fit`, its intercept a and r^2 reported): a is the
    curvature correction at these radii.

    Returns dict(sigma, sigma_fit, intercept, radii (equimolar), dp, rho_in,
    rho_out, fit_r2, steps)."""
    rl, rv = rho_guess
    Rs, dps, rins, routs, steps_all = [], [], [], [], []
    for R in radii:
        box = int(math.ceil(box_factor * R / 8.0) * 8)
        c = (box - 1) / 2.0
        g = np.arange(box) - c
        r = np.sqrt(g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2)
        rho0 = rv + 0.5 * (rl - rv) * (1.0 - np.tanh((r - R) / width))
        with _lattice((box, box, box), G, tau, collision, rates, storage, G2) as L:
            L.set_density(rho0)
            rho, steps = _run_to_steady(L, max_steps, check_every, tol)
        k = box // 2
        core = rho[k - 2:k + 2, k - 2:k + 2, k - 2:k + 2]  # the 4^3 cells around the centre
        rho_in = float(core.mean())
        rho_out = float(rho[0, 0, 0])  # the corner is farthest from the droplet
        V = float(box) ** 3
        Vl = (float(rho.sum()) - rho_out * V) / (rho_in - rho_out)
        Rs.append((3.0 * Vl / (4.0 * math.pi)) ** (1.0 / 3.0))
        dps.append(float(pressure(rho_in, G, G2=G2) - pressure(rho_out, G, G2=G2)))
        rins.append(rho_in)
        routs.append(rho_out)
        steps_all.append(steps)
    x = 1.0 / np.asarray(Rs)
    y = np.asarray(dps)
    slope, intercept = np.polyfit(x, y, 1)
    fit = slope * x + intercept
    ss = float(((y - y.mean()) ** 2).sum())
    r2 = 1.0 - float(((y - fit) ** 2).sum()) / ss if ss > 0 else 1.0
    return {"sigma": float((x * y).sum() / (x * x).sum() / 2.0), "sigma_fit": float(slope / 2.0),
            "intercept": float(intercept), "radii": Rs, "dp": dps,
            "rho_in": rins, "rho_out": routs, "fit_r2": r2, "steps": steps_all}


def calibrate_tau(R0, measure, tau0, Oh=0.1, rel_tol=1e-3, max_iter=12):
    """Fixed-point iteration of Sec. 3: tau -> measure(tau) = (sigma, rho_l)
    -> tau_for_oh.  Stops when two consecutive sigma agree to rel_tol.
    Returns dict(tau, sigma, rho_l, iterations, history)."""
    tau = tau0
    hist = []
    sigma_prev = None
    for it in range(1, max_iter + 1):
        sigma, rho_l = measure(tau)
        hist.append((tau, sigma, rho_l))
        new_tau = tau_for_oh(Oh, sigma, rho_l, R0)
        if sigma_prev is not None and abs(sigma - sigma_prev) <= rel_tol * abs(sigma):
            return {"tau": tau, "sigma": sigma, "rho_l": rho_l, "iterations": it, "history": hist,
                    "tau_next": new_tau}
        sigma_prev = sigma
        tau = new_tau
    return {"tau": tau, "sigma": sigma, "rho_l": rho_l, "iterations": max_iter, "history": hist,
            "tau_next": new_tau, "converged": False}
