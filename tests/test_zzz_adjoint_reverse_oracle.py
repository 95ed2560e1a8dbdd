"""The GPU adjoint's whole gradient field against the reverse-mode FP64
reference (oracle/reverse.py: the SRT step in PyTorch CPU ops, reversed by
torch.autograd), element by element, on a tiny ligament."""

import numpy as np
import pytest

from oracle import reverse as rv
from paper_1905_09554_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CUDA device only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_09554_gb300 import lbm  # noqa: E402

G0, TAU0 = -5.5, 0.9
RL, RV = inputs.COEXISTENCE[("shift", -5.5, 1.0)]


def neck_energy_grad(rho):
    """dJ/drho of J = mean_z (R(z) - mean R)^2, R = sqrt(A/pi),
    A(z) = sum_xy (rho - rho_v)/(rho_l - rho_v)."""
    nz = rho.shape[0]
    A = ((rho - RV) / (RL - RV)).sum(axis=(1, 2))
    R = np.sqrt(A / np.pi)
    g = (2.0 / nz) * (R - R.mean()) / (2.0 * np.pi * R * (RL - RV))
    return np.broadcast_to(g[:, None, None], rho.shape).copy()


@pytest.mark.parametrize("box,R0,steps,every", [((12, 12, 20), 3.0, 30, 7), ((16, 16, 32), 4.0, 40, 9)])
def test_adjoint_field_matches_the_reverse_mode_oracle(box, R0, steps, every):
    """12 x 12 x 20, and the 16 x 16 x 32 check size of the adjoint form."""
    rho0 = inputs.noisy_ligament_density(*box, R0, 0.1, RL, RV, 1e-3, seed=31)
    nz, ny, nx = rho0.shape
    with lbm.Lattice(nx, ny, nz, G=G0, tau=TAU0, storage="f64") as L:
        L.adjoint_forward(rho0, steps, every)
        r, _ = L.moments()
        g, gG, gT = L.adjoint_backward(neck_energy_grad(r))
    J_ref, g_ref, gG_ref, gT_ref = rv.gradient(rho0, G0, TAU0, steps, "neck", RL, RV)
    scale = np.abs(g_ref).max()
    assert np.abs(g - g_ref).max() <= 1e-9 * scale, np.abs(g - g_ref).max() / scale
    assert abs(gG - gG_ref) <= 1e-9 * max(1e-6, abs(gG_ref)), (gG, gG_ref)
    assert abs(gT - gT_ref) <= 1e-9 * max(1e-6, abs(gT_ref)), (gT, gT_ref)


def test_torch_rollout_misfit_gradient_matches_the_reverse_mode_oracle():
    """The density L2 misfit through paper_1905_09554_gb300.autograd.rollout
    (FP64 storage) against the reverse-mode oracle, whole field."""
    from paper_1905_09554_gb300 import autograd as lag

    rho0_np = inputs.noisy_ligament_density(12, 12, 20, 3.0, 0.1, RL, RV, 1e-3, seed=31)
    target = inputs.noisy_ligament_density(12, 12, 20, 3.3, 0.05, RL, RV, 1e-3, seed=4)
    steps = 20
    rho0 = torch.tensor(rho0_np, device="cuda", requires_grad=True)
    G = torch.tensor(G0, dtype=torch.float64, requires_grad=True)
    tau = torch.tensor(TAU0, dtype=torch.float64, requires_grad=True)
    rho_T = lag.rollout(rho0, G, tau, steps, every=5, storage="f64")
    J = 0.5 * ((rho_T - torch.tensor(target, device="cuda")) ** 2).sum()
    J.backward()
    J_ref, g_ref, gG_ref, gT_ref = rv.gradient(rho0_np, G0, TAU0, steps, "misfit", target=target)
    assert abs(J.item() - J_ref) <= 1e-12 * J_ref
    g = rho0.grad.cpu().numpy()
    assert np.abs(g - g_ref).max() <= 1e-9 * np.abs(g_ref).max()
    assert abs(G.grad.item() - gG_ref) <= 1e-9 * max(1e-6, abs(gG_ref))
    assert abs(tau.grad.item() - gT_ref) <= 1e-9 * max(1e-6, abs(gT_ref))
