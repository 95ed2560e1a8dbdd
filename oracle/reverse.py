"""Reverse-mode FP64 CPU reference for the gradient of a ligament objective
through n SRT steps with respect to the initial density field, G and tau.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: imported only by
tests.  It restates the SRT step of ``lbm_oracle`` (Sec. 2: psi law,
Eq. SC_force, Eq. local_eq, Eq. vel_shift, Eq. LBE) in plain PyTorch CPU
float64 ops and lets ``torch.autograd`` (a library primitive) run the
reverse pass, so the whole gradient field dJ/drho0(x) comes out of one
backward sweep.  No blocking, fusion or hand-derived adjoint: the forward is
the definition, the reverse is the library's chain rule.

The initial state is the rest equilibrium f = w rho0 (u = 0), as
``lbm_oracle.init_populations``.  Arrays: (nz, ny, nx), x fastest.
"""

from __future__ import annotations

import math

import torch

from . import lbm_oracle as o

_C = torch.tensor(o.C, dtype=torch.float64)  # (19, 3)
_W = torch.tensor(o.W, dtype=torch.float64)  # (19,)
_CS2 = o.CS2


def _shift(a, d):
    """a[x + d] for every x, periodic (the oracle's at_offset)."""
    dx, dy, dz = (int(v) for v in d)
    return torch.roll(a, shifts=(-dz, -dy, -dx), dims=(0, 1, 2))


def srt_step(f, G, tau, rho0=1.0):
    """One SRT step with the velocity shift: collide then push-stream."""
    rho = f.sum(dim=0)
    j = torch.einsum("qi,qzyx->izyx", _C, f)
    psi = rho0 * (1.0 - torch.exp(-rho / rho0))
    acc = torch.zeros((3,) + tuple(rho.shape), dtype=f.dtype)
    for a in range(o.Q):
        if not o.C[a].any():
            continue
        sh = _shift(psi, o.C[a])
        acc = acc + torch.stack([_W[a] * float(o.C[a][i]) * sh for i in range(3)])
    F = -G * psi * acc
    u = (j + tau * F) / rho
    cu = torch.einsum("qi,izyx->qzyx", _C, u)
    uu = (u * u).sum(dim=0)
    feq = _W.view(-1, 1, 1, 1) * rho * (1.0 + cu / _CS2 + cu * cu / (2 * _CS2 * _CS2) - uu / (2 * _CS2))
    fstar = f - (f - feq) / tau
    out = []
    for a in range(o.Q):
        dx, dy, dz = (int(v) for v in o.C[a])
        out.append(torch.roll(fstar[a], shifts=(dz, dy, dx), dims=(0, 1, 2)))
    return torch.stack(out)


def rollout(rho0, G, tau, steps):
    """Density after `steps` SRT steps from rest at density rho0 (tensors)."""
    f = _W.view(-1, 1, 1, 1) * rho0
    for _ in range(steps):
        f = srt_step(f, G, tau)
    return f.sum(dim=0)


def neck_energy(rho, rho_l, rho_v):
    """J = mean_z (R(z) - mean R)^2 with R(z) = sqrt(A(z)/pi) and the
    unclamped liquid area A(z) = sum_xy (rho - rho_v)/(rho_l - rho_v)."""
    A = ((rho - rho_v) / (rho_l - rho_v)).sum(dim=(1, 2))
    R = torch.sqrt(A / math.pi)
    return ((R - R.mean()) ** 2).mean()


def total_mass(rho):
    return rho.sum()


def misfit(rho, target):
    """Density L2 misfit J = sum (rho - target)^2 / 2."""
    return 0.5 * ((rho - target) ** 2).sum()


def gradient(rho0, G, tau, steps, objective="neck", rho_l=None, rho_v=None, target=None):
    """(J, dJ/drho0 as a numpy (nz, ny, nx) array, dJ/dG, dJ/dtau) of the
    objective ("neck": neck_energy with rho_l, rho_v; "mass": total mass;
    "misfit": L2 misfit against `target`) of the density after `steps` SRT
    steps from rest at rho0 (numpy)."""
    r0 = torch.tensor(rho0, dtype=torch.float64, requires_grad=True)
    g = torch.tensor(float(G), dtype=torch.float64, requires_grad=True)
    t = torch.tensor(float(tau), dtype=torch.float64, requires_grad=True)
    rho = rollout(r0, g, t, steps)
    if objective == "neck":
        J = neck_energy(rho, rho_l, rho_v)
    elif objective == "mass":
        J = total_mass(rho)
    elif objective == "misfit":
        J = misfit(rho, torch.tensor(target, dtype=torch.float64))
    else:
        raise ValueError(objective)
    J.backward()
    return float(J.detach()), r0.grad.numpy().copy(), float(g.grad), float(t.grad)
