"""Closed-form and continuum results used to pin the FP64 reference step.

TEST INFRASTRUCTURE ONLY (imported by ``tests/`` and the scripts under tests/golden/,
never by the library).  Nothing here runs the lattice; each function is a
textbook or continuum statement that the lattice results are compared with.
"""

from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize, special

CS2 = 1.0 / 3.0


def psi(rho, rho0=1.0):
    """Pseudo-potential of Sec. 2: rho0 (1 - exp(-rho/rho0))."""
    return rho0 * (1.0 - np.exp(-rho / rho0))


def dpsi(rho, rho0=1.0):
    return np.exp(-rho / rho0)


def eos(rho, G, rho0=1.0):
    """Non-ideal EoS of Eq. EOS_SC: P = rho cs2 + cs2 G psi^2 / 2."""
    return rho * CS2 + 0.5 * CS2 * G * psi(rho, rho0) ** 2


def coexistence_integral(G, eps, rho0=1.0, guess=(2.2, 0.08)):
    """Flat-interface coexistence densities from the continuum mechanical
    stability condition of the single-belt Shan-Chen model,
        P(rho_l) = P(rho_v) = p0,
        int_{rho_v}^{rho_l} (p0 - P(rho)) psi'(rho) / psi(rho)^(1+eps) drho = 0,
    with eps = 0 for the exact-difference (Guo-like) forcing and eps = 1 for
    the classic velocity-shift forcing at tau = 1 (Shan & Chen 1993/94;
    Shan 2008).  Solved to ~1e-12 by quadrature + Newton.  Returns (rho_l, rho_v).
    """
    def eqs(v):
        rl, rv = v
        p0 = eos(rv, G, rho0)
        g = lambda r: (p0 - eos(r, G, rho0)) * dpsi(r, rho0) / psi(r, rho0) ** (1.0 + eps)
        I, _ = integrate.quad(g, rv, rl, epsabs=1e-14, epsrel=1e-13, limit=200)
        return [eos(rl, G, rho0) - p0, I]

    sol = optimize.fsolve(eqs, guess, xtol=1e-13, full_output=True)
    rl, rv = sol[0]
    # fsolve returns its last iterate even when it did not converge: accept
    # only a solution with two distinct phases that satisfies both equations
    res = eqs((rl, rv))
    if not (rl > rv > 0) or max(abs(res[0]), abs(res[1])) > 1e-9:
        raise RuntimeError(f"coexistence_integral: no solution near {guess} (G = {G}, eps = {eps})")
    return float(rl), float(rv)


def rayleigh_inviscid(x):
    """Rayleigh (1878) growth rate of an inviscid liquid cylinder in vacuum,
    in units of 1/t_cap (t_cap = sqrt(rho_l R0^3 / sigma), Eq. Oh_Tcap):
        omega^2 = x I1(x)/I0(x) (1 - x^2),  x = k R0."""
    return math.sqrt(max(x * (1 - x * x) * special.iv(1, x) / special.iv(0, x), 0.0))


def viscous_long_wave(x, Oh):
    """One-dimensional (slender-jet) viscous growth rate in 1/t_cap:
    omega^2 + 3 Oh x^2 omega = x^2 (1 - x^2) / 2 (Eggers & Dupont 1994)."""
    b = 3.0 * Oh * x * x
    c = 0.5 * x * x * (1.0 - x * x)
    return 0.5 * (-b + math.sqrt(b * b + 4.0 * c))


def viscous_cylinder(x, Oh):
    """Growth rate (1/t_cap) of the linear Rayleigh-Plateau instability of a
    viscous liquid cylinder in vacuum, the relation of Chandrasekhar (1961),
    written from its derivation: with y^2 = x^2 + omega/Oh,
      omega^2 + 2 Oh x^2 omega [ I1'(x)/I0(x)
            - (2xy/(x^2+y^2)) (I1(x)/I0(x)) (I1'(y)/I1(y)) ]
        = x (1 - x^2) (I1(x)/I0(x)) (y^2 - x^2)/(y^2 + x^2).
    Returns 0 for stable wavenumbers (x >= 1)."""
    if x >= 1.0:
        return 0.0
    r1 = special.iv(1, x) / special.iv(0, x)

    def resid(w):
        y = math.sqrt(x * x + w / Oh)
        # I1'(y)/I1(y) = I0(y)/I1(y) - 1/y, from exponentially scaled Bessels
        ry = special.ive(0, y) / special.ive(1, y) - 1.0 / y
        br = (special.ivp(1, x) / special.iv(0, x)
              - (2 * x * y / (x * x + y * y)) * r1 * ry)
        return w * w + 2 * Oh * x * x * w * br - x * (1 - x * x) * r1 * (y * y - x * x) / (y * y + x * x)

    hi = rayleigh_inviscid(x) + 1e-9
    return optimize.brentq(resid, 1e-14, hi, xtol=1e-15)


def linear_breakup_time(eps, omega):
    """Linear estimate of the break-up time (Sec. 4): the perturbation
    eps R0 grows as exp(omega t) and breaks the ligament at amplitude R0, so
    T = ln(1/eps) / omega (in the units of 1/omega)."""
    return math.log(1.0 / eps) / omega
