"""torch.autograd access to the discrete adjoint of the SRT step.

``rollout(rho0, G, tau, n)`` runs n steps of the Shan-Chen SRT lattice from
rest with density rho0 (a float64 CUDA tensor of shape (nz, ny, nx)) and
returns the density rho(n).  Any torch objective of rho(n) can then be
differentiated with respect to rho0, G and tau: the backward pass calls the
library's adjoint kernels (lbm_adjoint_backward), which recompute the forward
states from checkpoints kept every ``every`` steps (default ~sqrt(n)).
"""

from __future__ import annotations

import math

import torch

from . import lbm


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, G, tau, n, every, storage, rho_ref):
        nz, ny, nx = rho0.shape
        L = lbm.Lattice(nx, ny, nz, G=float(G), tau=float(tau), collision="srt", storage=storage,
                        rho_ref=rho_ref)
        L.adjoint_forward(rho0.detach().to(torch.float64).contiguous(), n, every)
        rho_T = torch.empty((nz, ny, nx), dtype=torch.float64, device=rho0.device)
        L.moments_device(rho_T)
        ctx.lattice = L
        return rho_T

    @staticmethod
    def backward(ctx, g):
        L = ctx.lattice
        d_rho0 = torch.empty(g.shape, dtype=torch.float64, device=g.device)  # dense, x fastest
        _, dG, dtau = L.adjoint_backward(g.detach().to(torch.float64).contiguous(), out=d_rho0)
        torch.cuda.current_stream().synchronize()
        L.close()
        ctx.lattice = None
        dev = g.device
        return (d_rho0, torch.tensor(dG, dtype=torch.float64, device=dev),
                torch.tensor(dtau, dtype=torch.float64, device=dev), None, None, None, None)


def rollout(rho0: torch.Tensor, G, tau, n: int, every: int | None = None, storage: str = "f32",
            rho_ref: float = 1.0) -> torch.Tensor:
    """rho(n) after n SRT steps from rest with density rho0; differentiable in
    rho0, G and tau (pass tensors with requires_grad for the latter two)."""
    if every is None:
        every = max(1, int(round(math.sqrt(n))))
    G = G if isinstance(G, torch.Tensor) else torch.tensor(float(G), dtype=torch.float64)
    tau = tau if isinstance(tau, torch.Tensor) else torch.tensor(float(tau), dtype=torch.float64)
    return _Rollout.apply(rho0, G, tau, int(n), int(every), storage, float(rho_ref))


def neck_energy(rho: torch.Tensor, rho_l: float, rho_v: float) -> torch.Tensor:
    """Perturbation energy of the neck profile: with the liquid area of slice
    z, A(z) = sum_xy (rho - rho_v)/(rho_l - rho_v), and R(z) = sqrt(A(z)/pi),
    J = mean_z (R(z) - mean R)^2.  (The plain mean of R^2 is proportional to
    the conserved mass, so its gradient with respect to G and tau vanishes.)"""
    A = ((rho - rho_v) / (rho_l - rho_v)).sum(dim=(1, 2))
    R = torch.sqrt(A / math.pi)
    return ((R - R.mean()) ** 2).mean()
