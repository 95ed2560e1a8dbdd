"""A second, numpy-free restatement of the step (plain Python lists and
loops, `math.exp`) on tiny periodic boxes, against the numpy oracle.

It is written from the definitions, not from the oracle's code paths:
neighbours by explicit modular indexing instead of array rolls, the MRT
collision as a sum of projections on the orthogonal d'Humieres moments
(f* = f + sum_k M_k [ -s_k (m_k - m_k^eq) + (1 - s_k / 2) (M S)_k ] / |M_k|^2)
instead of a matrix inverse, the Guo source and the equilibrium per cell
and per velocity.  A sign, index or transposition slip on either side makes
them disagree.  CPU only.
"""

import math
import random

import numpy as np
import pytest

from oracle import lbm_oracle as o

# D3Q19 in its own order here (rest, 6 axis, 12 edge vectors)
VEL = [(0, 0, 0)]
VEL += [(s, 0, 0) for s in (1, -1)] + [(0, s, 0) for s in (1, -1)] + [(0, 0, s) for s in (1, -1)]
VEL += [(a, b, 0) for a in (1, -1) for b in (1, -1)]
VEL += [(a, 0, b) for a in (1, -1) for b in (1, -1)]
VEL += [(0, a, b) for a in (1, -1) for b in (1, -1)]
WGT = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12


def moment_rows():
    """The 19 d'Humieres D3Q19 moments as polynomials of c, in the order
    rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz,
    mx, my, mz."""
    def polys(c):
        x, y, z = c
        c2 = x * x + y * y + z * z
        return [1, 19 * c2 - 30, (21 * c2 * c2 - 53 * c2 + 24) / 2,
                x, (5 * c2 - 9) * x, y, (5 * c2 - 9) * y, z, (5 * c2 - 9) * z,
                3 * x * x - c2, (3 * c2 - 5) * (3 * x * x - c2),
                y * y - z * z, (3 * c2 - 5) * (y * y - z * z),
                x * y, y * z, x * z,
                (y * y - z * z) * x, (z * z - x * x) * y, (x * x - y * y) * z]
    cols = [polys(c) for c in VEL]
    return [[cols[a][k] for a in range(19)] for k in range(19)]


ROWS = moment_rows()
NORM = [sum(v * v for v in row) for row in ROWS]


def psi_of(r):
    return 1.0 - math.exp(-r)


def feq(rho, u):
    out = []
    uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    for c, w in zip(VEL, WGT):
        cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2]
        out.append(w * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu))
    return out


def plain_step(f, dims, G, coll, tau, s):
    """f[z][y][x][a] -> the next step's populations, same layout."""
    nx, ny, nz = dims
    rho = [[[sum(f[z][y][x]) for x in range(nx)] for y in range(ny)] for z in range(nz)]
    new = [[[[0.0] * 19 for _ in range(nx)] for _ in range(ny)] for _ in range(nz)]
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                cell = f[z][y][x]
                r = rho[z][y][x]
                j = [sum(c[i] * fa for c, fa in zip(VEL, cell)) for i in range(3)]
                acc = [0.0, 0.0, 0.0]
                for c, w in zip(VEL, WGT):
                    nb = rho[(z + c[2]) % nz][(y + c[1]) % ny][(x + c[0]) % nx]
                    for i in range(3):
                        acc[i] += w * psi_of(nb) * c[i]
                F = [-G * psi_of(r) * acc[i] for i in range(3)]
                if coll == "srt":
                    ushift = [(j[i] + tau * F[i]) / r for i in range(3)]
                    eq = feq(r, ushift)
                    post = [cell[a] - (cell[a] - eq[a]) / tau for a in range(19)]
                else:
                    ub = [(j[i] + 0.5 * F[i]) / r for i in range(3)]
                    eq = feq(r, ub)
                    S = []
                    for c, w in zip(VEL, WGT):
                        cu = sum(c[i] * ub[i] for i in range(3))
                        S.append(w * sum((3 * (c[i] - ub[i]) + 9 * cu * c[i]) * F[i] for i in range(3)))
                    post = list(cell)
                    for k in range(19):
                        m = sum(ROWS[k][a] * cell[a] for a in range(19))
                        me = sum(ROWS[k][a] * eq[a] for a in range(19))
                        ms = sum(ROWS[k][a] * S[a] for a in range(19))
                        d = -s[k] * (m - me) + (1 - 0.5 * s[k]) * ms
                        for a in range(19):
                            post[a] += ROWS[k][a] * d / NORM[k]
                for a, c in enumerate(VEL):
                    new[(z + c[2]) % nz][(y + c[1]) % ny][(x + c[0]) % nx][a] = post[a]
    return new


def to_numpy(f, dims):
    """Plain layout -> the oracle's (19, nz, ny, nx) in its own velocity order."""
    nx, ny, nz = dims
    out = np.empty((19, nz, ny, nx))
    for q, c in enumerate(o.C):
        a = VEL.index(tuple(int(v) for v in c))
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    out[q, z, y, x] = f[z][y][x][a]
    return out


@pytest.mark.parametrize("coll,tau", [("srt", 1.0), ("srt", 0.7), ("mrt", 0.8), ("mrt", 1.3)])
def test_plain_python_step_matches_the_numpy_oracle(coll, tau):
    dims = (3, 4, 5)
    nx, ny, nz = dims
    rng = random.Random(17)
    G = -5.5
    # random density with a random small velocity per cell, as equilibria
    f = [[[feq(rng.uniform(0.2, 2.2), [rng.uniform(-0.05, 0.05) for _ in range(3)]) for _ in range(nx)]
          for _ in range(ny)] for _ in range(nz)]
    s = [rng.uniform(0.6, 1.8) for _ in range(19)] if coll == "mrt" else None
    f_np = to_numpy(f, dims)
    # rates follow the oracle's moment order, which is the one used here
    p = o.Params(G=G, tau=tau, collision=coll, s=np.array(s) if s else None)
    for _ in range(2):
        f = plain_step(f, dims, G, coll, tau, s)
        f_np = o.step(f_np, p)
    assert np.abs(to_numpy(f, dims) - f_np).max() < 1e-13
