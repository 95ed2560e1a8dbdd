"""Two-belt (multirange) pseudo-potential force: the extension of the
Shan-Chen force that Sec. 2 of the paper names (its refs. to Sbragaglia et
al. and Falcucci et al.) as the way to tune the surface tension independently
of the equation of state, and does not run.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: plain numpy and exact
rational arithmetic, imported only by tests.

The paper prints no formula for it; the reading used here:

    F(x) = -psi(x) [ G1 sum_{a in D3Q19} w_a psi(x + c_a) c_a
                   + G2 sum_{b in E8}   (p_b / 3) psi(x + e_b) e_b ]

* belt 1 is the single-belt force of Eq. SC_force (D3Q19 vectors, lattice
  weights w, second moment sum_a w_a c_ax^2 = cs2 = 1/3);
* belt 2 runs over E8: the 92 vectors with components in {-2..2} and
  |e|^2 in {1, 2, 3, 4, 5, 6, 8}, with one weight p per shell, the unique set
  with sum_b p_b e_bx^2 = 1 whose moment tensors are isotropic up to eighth
  order (`e8_weights` solves for it exactly); the factor 1/3 gives it the
  same second moment as belt 1.

So for slowly varying psi, F = -cs2 (G1 + G2) psi grad psi + O(grad^3): the
bulk equation of state is P = rho cs2 + cs2 (G1 + G2) psi^2 / 2, while the
third-order terms, which set the surface tension, weigh the two belts
differently.  G2 = 0 is Eq. SC_force.
"""

from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np

from . import lbm_oracle as o

E8_SHELLS = (1, 2, 3, 4, 5, 6, 8)


def e8_vectors():
    """The 92 integer vectors with components in {-2..2} and |e|^2 in E8_SHELLS,
    as an int array (92, 3)."""
    vecs = [v for v in itertools.product(range(-2, 3), repeat=3) if sum(a * a for a in v) in E8_SHELLS]
    return np.array(vecs, dtype=np.int64)


def _shell_moment(shell, ex, ey, ez):
    """sum over the vectors of one shell of x^ex y^ey z^ez (an integer)."""
    tot = 0
    for v in itertools.product(range(-2, 3), repeat=3):
        if sum(a * a for a in v) == shell:
            tot += v[0] ** ex * v[1] ** ey * v[2] ** ez
    return tot


def _solve_exact(A, b):
    """Gauss-Jordan elimination over the rationals."""
    n = len(b)
    M = [[Fraction(x) for x in row] + [Fraction(bb)] for row, bb in zip(A, b)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [x / pv for x in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                fac = M[r][col]
                M[r] = [x - fac * y for x, y in zip(M[r], M[col])]
    return [M[r][n] for r in range(n)]


def e8_weights():
    """Weights p by shell (dict shell -> Fraction): normalisation
    sum p e_x^2 = 1 and isotropy of the 4th, 6th and 8th moment tensors.  For
    shells closed under the cube group, isotropy reduces to ratios of the
    moments <x^a y^b z^c> = sum p x^a y^b z^c: 4th order <x^4> = 3 <x^2 y^2>;
    6th order <x^6> = 15 <x^2y^2z^2>, <x^4 y^2> = 3 <x^2y^2z^2>; 8th order
    <x^8> : <x^6 y^2> : <x^4 y^4> : <x^4 y^2 z^2> = 105 : 15 : 9 : 3."""
    S = E8_SHELLS

    def row(ex, ey, ez):
        return [_shell_moment(s, ex, ey, ez) for s in S]

    def diff(r1, k1, r2, k2):  # k1 * r1 - k2 * r2 = 0
        return [k1 * a - k2 * b for a, b in zip(r1, r2)]

    A = [row(2, 0, 0)]
    b = [1]
    A.append(diff(row(4, 0, 0), 1, row(2, 2, 0), 3)); b.append(0)
    A.append(diff(row(6, 0, 0), 1, row(2, 2, 2), 15)); b.append(0)
    A.append(diff(row(4, 2, 0), 1, row(2, 2, 2), 3)); b.append(0)
    A.append(diff(row(8, 0, 0), 3, row(4, 2, 2), 105)); b.append(0)
    A.append(diff(row(6, 2, 0), 3, row(4, 2, 2), 15)); b.append(0)
    A.append(diff(row(4, 4, 0), 3, row(4, 2, 2), 9)); b.append(0)
    p = _solve_exact(A, b)
    return dict(zip(S, p))


E8 = e8_vectors()
_P = e8_weights()
P8 = np.array([float(_P[int((v * v).sum())]) for v in E8])  # weight of each vector


def belt_sum(psi, vecs, weights):
    """sum_b weights_b psi(x + e_b) e_b, shape (3, nz, ny, nx)."""
    acc = np.zeros((3,) + psi.shape, dtype=np.result_type(psi, np.float64))
    for v, wgt in zip(vecs, weights):
        if not v.any():
            continue
        shifted = o.at_offset(psi, v)
        for i in range(3):
            if v[i] != 0:
                acc[i] += wgt * v[i] * shifted
    return acc


def two_belt_force(rho, G1, G2, rho0=1.0):
    """F = -psi(x) [G1 (D3Q19 belt) + G2 (E8 belt, weights p/3)], periodic."""
    psi = o.pseudo_potential(rho, rho0)
    acc = G1 * belt_sum(psi, o.C, o.W)
    if G2 != 0:
        acc = acc + G2 * belt_sum(psi, E8, P8 / 3.0)
    return -psi * acc


def pressure(rho, G1, G2, rho0=1.0):
    """Bulk pressure: rho cs2 + cs2 (G1 + G2) psi^2 / 2."""
    return rho * o.CS2 + 0.5 * o.CS2 * (G1 + G2) * o.pseudo_potential(rho, rho0) ** 2


def collide(f, p, G2):
    """One collision of `p` (an lbm_oracle.Params) with the two-belt force."""
    F = two_belt_force(o.density(f), p.G, G2, p.rho0)
    if p.collision == "srt":
        return o.collide_srt(f, F, p.tau)
    return o.collide_mrt(f, F, p.s)


def run(f, n, p, G2):
    for _ in range(n):
        f = o.stream(collide(f, p, G2))
    return f


def macroscopic(f, p, G2):
    rho = o.density(f)
    F = two_belt_force(rho, p.G, G2, p.rho0)
    return rho, (o.momentum(f) + 0.5 * F) / rho
