"""Plain FP64 CPU reference of the pseudo-potential (Shan-Chen) D3Q19 lattice
Boltzmann step of Chiappini, Xue, Falcucci, Sbragaglia, "Hydrodynamic behavior
of the Pseudo-Potential lattice Boltzmann method for interfacial flows"
(arXiv:1905.09554).

TEST INFRASTRUCTURE ONLY.  This module is the oracle that the CUDA path is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the library never does.  It shares
no code, table or helper with the CUDA sources.

Everything is numpy, float64 (complex128 also flows through every function, so
complex-step derivatives of the whole step are available), written in the order
and notation of Sec. 2 of the paper, without blocking or fusion:

* the lattice (Sec. 2, "D3Q19"): velocities and weights;
* moments (Eq. momentum);
* pseudo-potential psi = rho0 (1 - exp(-rho/rho0)) and the single-belt
  Shan-Chen force (Eq. SC_force);
* equilibrium (Eq. local_eq, with the leading "1 +" restored);
* SRT collision with the velocity shift (Eq. vel_shift);
* MRT collision with Guo-like forcing and the barycentric velocity
  (Eq. barycentric), d'Humieres D3Q19 moment basis;
* periodic streaming (Eq. LBE);
* the EoS (Eq. EOS_SC) and diagnostics used by the physics checks.

Readings of passages that are garbled or silent are listed in the project's
design notes; each function states the one it uses.

Arrays: a field is (nz, ny, nx) with x fastest; populations are (19, nz, ny, nx).
"""

from __future__ import annotations

import itertools
import math

import numpy as np

CS2 = 1.0 / 3.0  # squared lattice speed of sound (Sec. 2)


# --------------------------------------------------------------------------
# Lattice (Sec. 2): D3Q19 = the 19 vectors of {-1,0,1}^3 with |c|^2 <= 2.
# Weights by speed shell: 1/3 (rest), 1/18 (|c|^2 = 1), 1/36 (|c|^2 = 2).
# --------------------------------------------------------------------------
def d3q19():
    """Return (c, w): c int array (19, 3) of (cx, cy, cz), w float64 (19,)."""
    shell_weight = {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}
    vecs = [v for v in itertools.product((0, 1, -1), repeat=3)
            if sum(abs(a) for a in v) <= 2]
    c = np.array(vecs, dtype=np.int64)
    w = np.array([shell_weight[int((v * v).sum())] for v in c])
    return c, w


C, W = d3q19()
Q = len(W)


def at_offset(a, d):
    """Field value at x + d for every x, periodic: out[x] = a[x + d]."""
    dx, dy, dz = (int(v) for v in d)
    return np.roll(a, shift=(-dz, -dy, -dx), axis=(0, 1, 2))


# --------------------------------------------------------------------------
# Moments (Eq. momentum)
# --------------------------------------------------------------------------
def density(f):
    return f.sum(axis=0)


def momentum(f):
    """j = sum_a c_a f_a, shape (3, nz, ny, nx) ordered (jx, jy, jz)."""
    return np.tensordot(C.T.astype(np.float64), f, axes=(1, 0))


# --------------------------------------------------------------------------
# Pseudo-potential and Shan-Chen force (Eq. SC_force and the psi law after it)
# --------------------------------------------------------------------------
def pseudo_potential(rho, rho0=1.0):
    return rho0 * (1.0 - np.exp(-rho / rho0))


def shan_chen_force(rho, G, rho0=1.0):
    """F(x) = -G psi(x) sum_a w_a psi(x + c_a) c_a (single belt, periodic).
    The rest vector contributes nothing (c_0 = 0).  Shape (3, nz, ny, nx)."""
    psi = pseudo_potential(rho, rho0)
    acc = np.zeros((3,) + rho.shape, dtype=np.result_type(rho, np.float64))
    for a in range(Q):
        if not C[a].any():
            continue
        shifted = at_offset(psi, C[a])
        for i in range(3):
            if C[a][i] != 0:
                acc[i] += W[a] * C[a][i] * shifted
    return -G * psi * acc


# --------------------------------------------------------------------------
# Equilibrium (Eq. local_eq).  The printed bracket lacks its leading 1; without
# it sum_a f_eq != rho, so the reading is the standard second-order Maxwellian
#   f_eq_a = w_a rho [1 + c.u/cs2 + (c.u)^2/(2 cs2^2) - u.u/(2 cs2)].
# --------------------------------------------------------------------------
def equilibrium(rho, u):
    cu = np.tensordot(C.astype(np.float64), u, axes=(1, 0))  # (19, ...)
    uu = (u * u).sum(axis=0)
    wr = W.reshape((Q,) + (1,) * rho.ndim) * rho
    return wr * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2))


# --------------------------------------------------------------------------
# SRT with shifted equilibrium (Eq. LBE with Omega = dt/tau, Eq. vel_shift).
# "u" in Eq. vel_shift is read as the bare velocity j/rho.
# --------------------------------------------------------------------------
def collide_srt(f, F, tau):
    rho = density(f)
    u = momentum(f) / rho
    u_shift = u + tau * F / rho
    return f - (f - equilibrium(rho, u_shift)) / tau


# --------------------------------------------------------------------------
# MRT (Eq. LBE with Omega = M^-1 Lambda M; the paper prints M Lambda M^-1, the
# standard operator order is used).  Basis: d'Humieres et al. (2002) D3Q19,
# moments (0-based)
#   0 rho, 1 e, 2 eps, 3 jx, 4 qx, 5 jy, 6 qy, 7 jz, 8 qz, 9 3pxx, 10 3pixx,
#   11 pww, 12 piww, 13 pxy, 14 pyz, 15 pxz, 16 mx, 17 my, 18 mz.
# --------------------------------------------------------------------------
def mrt_matrix():
    rows = []
    cx, cy, cz = (C[:, i].astype(np.float64) for i in range(3))
    c2 = cx * cx + cy * cy + cz * cz
    rows.append(np.ones(Q))
    rows.append(19.0 * c2 - 30.0)
    rows.append((21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0)
    rows.append(cx)
    rows.append((5.0 * c2 - 9.0) * cx)
    rows.append(cy)
    rows.append((5.0 * c2 - 9.0) * cy)
    rows.append(cz)
    rows.append((5.0 * c2 - 9.0) * cz)
    rows.append(3.0 * cx * cx - c2)
    rows.append((3.0 * c2 - 5.0) * (3.0 * cx * cx - c2))
    rows.append(cy * cy - cz * cz)
    rows.append((3.0 * c2 - 5.0) * (cy * cy - cz * cz))
    rows.append(cx * cy)
    rows.append(cy * cz)
    rows.append(cx * cz)
    rows.append((cy * cy - cz * cz) * cx)
    rows.append((cz * cz - cx * cx) * cy)
    rows.append((cx * cx - cy * cy) * cz)
    return np.array(rows)


M = mrt_matrix()
M_INV = np.linalg.inv(M)


def mrt_rates(tau, rule="paper", s_other=1.0):
    """Diagonal of Lambda.  Sec. 2 sets s2 = s10 = s12 = s14 = s15 = s16 = omega
    (1-based), all others 1.  The printed omega = 2cs2/(cs2 + nu) is read as
    the standard omega = 2cs2/(cs2 + 2 nu) = 1/tau with nu = cs2 (tau - 1/2).

    rule "paper": the energy (bulk) moment and the five shear moments relax at
    1/tau, all others at ``s_other``.  rule "shear": only the five shear moments
    at 1/tau, bulk and ghosts at ``s_other``."""
    s = np.full(Q, float(s_other))
    omega = 1.0 / tau
    shear = [9, 11, 13, 14, 15]
    for k in shear:
        s[k] = omega
    if rule == "paper":
        s[1] = omega
    elif rule != "shear":
        raise ValueError(rule)
    return s


def guo_source(u, F):
    """Guo forcing term in population space,
    S_a = w_a [3 (c_a - u) + 9 (c_a . u) c_a] . F  (shape (19, ...))."""
    Cf = C.astype(np.float64)
    cF = np.tensordot(Cf, F, axes=(1, 0))
    cu = np.tensordot(Cf, u, axes=(1, 0))
    uF = (u * F).sum(axis=0)
    wr = W.reshape((Q,) + (1,) * (F.ndim - 1))
    return wr * (3.0 * (cF - uF) + 9.0 * cu * cF)


def collide_mrt(f, F, s):
    """MRT with Guo-like forcing (Eq. barycentric):
    u_b = (j + F/2)/rho, m = M f, m_eq = M f_eq(rho, u_b),
    m* = m - Lambda (m - m_eq) + (I - Lambda/2) M S,  f* = M^-1 m*."""
    rho = density(f)
    ub = (momentum(f) + 0.5 * F) / rho
    feq = equilibrium(rho, ub)
    S = guo_source(ub, F)
    m = np.tensordot(M, f, axes=(1, 0))
    meq = np.tensordot(M, feq, axes=(1, 0))
    mS = np.tensordot(M, S, axes=(1, 0))
    sv = np.asarray(s, dtype=np.float64).reshape((Q,) + (1,) * rho.ndim)
    mstar = m - sv * (m - meq) + (1.0 - 0.5 * sv) * mS
    return np.tensordot(M_INV, mstar, axes=(1, 0))


# --------------------------------------------------------------------------
# Streaming (Eq. LBE): f_a(x + c_a, t + 1) = f*_a(x, t), periodic box.
# --------------------------------------------------------------------------
def stream(fstar):
    out = np.empty_like(fstar)
    for a in range(Q):
        dx, dy, dz = (int(v) for v in C[a])
        out[a] = np.roll(fstar[a], shift=(dz, dy, dx), axis=(0, 1, 2))
    return out


# --------------------------------------------------------------------------
# One time step.  Populations at step t are post-streaming, pre-collision.
# --------------------------------------------------------------------------
class Params:
    """collision: 'srt' (velocity shift) or 'mrt' (Guo-like forcing)."""

    def __init__(self, G=-5.5, tau=1.0, collision="srt", s=None, rho0=1.0):
        self.G = G
        self.tau = tau
        self.collision = collision
        self.rho0 = rho0
        self.s = mrt_rates(tau) if (s is None and collision == "mrt") else s


def collide(f, p: Params):
    F = shan_chen_force(density(f), p.G, p.rho0)
    if p.collision == "srt":
        return collide_srt(f, F, p.tau)
    if p.collision == "mrt":
        return collide_mrt(f, F, p.s)
    raise ValueError(p.collision)


def step(f, p: Params):
    return stream(collide(f, p))


def run(f, n, p: Params):
    for _ in range(n):
        f = step(f, p)
    return f


def init_populations(rho, u=None):
    """Populations at rest equilibrium f = f_eq(rho, u) (u = 0 by default)."""
    if u is None:
        u = np.zeros((3,) + rho.shape)
    return equilibrium(rho, u)


def macroscopic(f, p: Params):
    """rho and the reported velocity u_b = (j + F/2)/rho (Eq. barycentric),
    used for both collision operators."""
    rho = density(f)
    F = shan_chen_force(rho, p.G, p.rho0)
    return rho, (momentum(f) + 0.5 * F) / rho


# --------------------------------------------------------------------------
# EoS (Eq. EOS_SC): P = rho cs2 + cs2 G psi^2 / 2.
# --------------------------------------------------------------------------
def pressure(rho, G, rho0=1.0):
    return rho * CS2 + 0.5 * CS2 * G * pseudo_potential(rho, rho0) ** 2


# --------------------------------------------------------------------------
# Diagnostics of the ligament (neck radius, Sec. 4; break-up, Sec. 4).
# --------------------------------------------------------------------------
def slice_diagnostics(rho, rho_l, rho_v):
    """Per z slice: liquid area A(z) = sum_xy clamp((rho - rho_v)/(rho_l -
    rho_v), 0, 1) and max_xy rho.  Returns (A, maxrho), each (nz,)."""
    phi = np.clip((rho - rho_v) / (rho_l - rho_v), 0.0, 1.0)
    return phi.sum(axis=(1, 2)), rho.max(axis=(1, 2))


def equivalent_radius(area):
    return np.sqrt(area / math.pi)
