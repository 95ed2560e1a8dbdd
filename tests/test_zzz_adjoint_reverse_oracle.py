"""The GPU adjoint's whole gradient field against the reverse-mode FP64
reference (oracle/reverse.py: the SRT step in PyTorch CPU ops, reversed by
torch.autograd), element by element, on a tiny ligament."""

import numpy as np
import pytest

from oracle import reverse as rv
from paper_1905_09554_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - GPU machine only
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


def test_adjoint_field_matches_the_reverse_mode_oracle():
    rho0 = inputs.noisy_ligament_density(12, 12, 20, 3.0, 0.1, RL, RV, 1e-3, seed=31)
    steps = 30
    nz, ny, nx = rho0.shape
    with lbm.Lattice(nx, ny, nz, G=G0, tau=TAU0, storage="f64") as L:
        L.adjoint_forward(rho0, steps, 7)
        r, _ = L.moments()
        g, gG, gT = L.adjoint_backward(neck_energy_grad(r))
    J_ref, g_ref, gG_ref, gT_ref = rv.gradient(rho0, G0, TAU0, steps, "neck", RL, RV)
    scale = np.abs(g_ref).max()
    assert np.abs(g - g_ref).max() <= 1e-9 * scale, np.abs(g - g_ref).max() / scale
    assert abs(gG - gG_ref) <= 1e-9 * max(1e-6, abs(gG_ref)), (gG, gG_ref)
    assert abs(gT - gT_ref) <= 1e-9 * max(1e-6, abs(gT_ref)), (gT, gT_ref)
