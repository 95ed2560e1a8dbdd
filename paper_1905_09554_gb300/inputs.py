"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds the problem set-up only (Sec. 3, "Simulations set-up"): the
perturbed-ligament initial density, a counter-based Gaussian noise field and the
per-instance parameters of the batched workload.  It holds none of the lattice
Boltzmann step's arithmetic (no lattice tables, no equilibrium, no force, no
collision, no streaming), so that it can feed both sides of a parity test.

Layout convention for every field: a C-ordered float64 array of shape
(nz, ny, nx), x fastest; cell (x, y, z) is ``a[z, y, x]``.
"""

from __future__ import annotations

import math

import numpy as np

# Liquid/vapour coexistence densities of the flat interface, produced by the
# committed script ``tests/golden/make_coexistence.py`` (which runs the plain
# FP64 reference implementation to steady state) and stored in
# ``tests/golden/coexistence.json``.  Keyed by (forcing, G, tau).  They only set
# the end points of the initial tanh profile; nothing depends on them exactly.
COEXISTENCE = {
    ("shift", -5.5, 1.0): (2.306809, 0.104103),
    ("guo", -5.5, 1.0): (2.248703, 0.056949),
    ("shift", -5.3, 1.0): (2.161682, 0.121367),
    ("guo", -5.3, 1.0): (2.10895, 0.078116),
}

_MASK64 = (1 << 64) - 1


def splitmix64(counter: np.ndarray, seed: int) -> np.ndarray:
    """SplitMix64 (Steele, Lea, Flood 2014) evaluated at ``seed + counter``.

    Counter-based: output k depends only on (seed, k), so any side can
    regenerate any element.  Works on uint64 arrays with wrap-around.
    """
    with np.errstate(over="ignore"):
        z = (np.uint64(seed & _MASK64) + counter.astype(np.uint64)
             * np.uint64(0x9E3779B97F4A7C15) + np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(n: int, seed: int, offset: int = 0) -> np.ndarray:
    """n doubles in (0, 1): the top 53 bits of SplitMix64, shifted off zero."""
    k = np.arange(offset, offset + n, dtype=np.uint64)
    bits = splitmix64(k, seed) >> np.uint64(11)
    return (bits.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def gaussian(n: int, seed: int) -> np.ndarray:
    """n standard normal deviates by the Box-Muller transform (1958) of
    consecutive SplitMix64 uniform pairs."""
    m = (n + 1) // 2
    u = uniform01(2 * m, seed)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:n]


def ligament_density(nx: int, ny: int, nz: int, R0: float, eps: float,
                     rho_l: float, rho_v: float, width: float = 2.0,
                     n_waves: int = 1) -> np.ndarray:
    """Initial density of a liquid cylinder along z with a cosine-perturbed
    surface, R(z) = R0 (1 + eps cos(2 pi n_waves z / nz)) (Sec. 3; the paper
    perturbs along its x axis with two wavelengths, this set-up uses z).

    The axis passes through ((nx-1)/2, (ny-1)/2); r is the distance of the
    cell node from it.  The profile is
    rho = rho_v + (rho_l - rho_v)/2 * (1 - tanh((r - R(z)) / width)).
    Returns float64 (nz, ny, nx).
    """
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    xc, yc = 0.5 * (nx - 1), 0.5 * (ny - 1)
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    R = R0 * (1.0 + eps * np.cos(2.0 * math.pi * n_waves * z / nz))
    return rho_v + 0.5 * (rho_l - rho_v) * (1.0 - np.tanh((r - R) / width))


def noisy_ligament_density(nx, ny, nz, R0, eps, rho_l, rho_v, sigma, seed,
                           width=2.0):
    """Ligament density plus per-cell Gaussian amplitude noise sigma * xi,
    xi from :func:`gaussian` with the given seed (x fastest)."""
    rho = ligament_density(nx, ny, nz, R0, eps, rho_l, rho_v, width)
    return rho + sigma * gaussian(rho.size, seed).reshape(rho.shape)


def random_density(nx, ny, nz, seed, lo=0.1, hi=2.3):
    """Uniform random density field in [lo, hi) (x fastest); a rough two-phase
    stress input for parity tests."""
    u = uniform01(nx * ny * nz, seed).reshape(nz, ny, nx)
    return lo + (hi - lo) * u


def ligament_box(R0: float, kR0: float, mode: str = "ceil"):
    """Box 4R0 x 4R0 x L for one wavelength L = 2 pi R0 / kR0 along z.
    ``mode`` rounds L up ('ceil') or to nearest ('round')."""
    L = 2.0 * math.pi * R0 / kR0
    nz = int(math.ceil(L - 1e-9)) if mode == "ceil" else int(round(L))
    n = int(round(4 * R0))
    return n, n, nz


def batch_instances(n: int = 64, seed: int = 0, radii=(8, 12, 16),
                    k_lo: float = 0.2, k_hi: float = 1.0):
    """Independent ligaments of uneven size: R0 drawn from ``radii`` and kR0
    uniform on [k_lo, k_hi), both from SplitMix64 with ``seed``.  Each gets a
    periodic box 4R0 x 4R0 x round(2 pi R0 / kR0).  Returns a list of dicts."""
    u = uniform01(2 * n, seed)
    out = []
    for i in range(n):
        R0 = float(radii[min(int(u[2 * i] * len(radii)), len(radii) - 1)])
        kR0 = k_lo + (k_hi - k_lo) * float(u[2 * i + 1])
        nx, ny, nz = ligament_box(R0, kR0, mode="round")
        out.append(dict(R0=R0, kR0=kR0, nx=nx, ny=ny, nz=nz))
    return out
