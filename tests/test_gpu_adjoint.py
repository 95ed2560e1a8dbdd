"""Discrete adjoint of the SRT step (lbm_adjoint_forward/backward and the
torch.autograd wrapper).

* Against the FP64 reference: complex-step derivatives of the reference
  rollout (exact to rounding, no adjoint derivation involved) for the
  gradient with respect to rho0 (along random directions), G and tau.
* Against central finite differences of the GPU FP64 forward (h = 1e-4).
* Checkpoint interval never changes a bit; the FP32 adjoint agrees with the
  FP64 one to FP32 accuracy.
* A conserved objective (total mass) has the exact gradient 1, 0, 0.
"""

import math

import numpy as np
import pytest

from oracle import lbm_oracle as o
from paper_1905_09554_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CUDA device only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_09554_gb300 import autograd as lag  # noqa: E402
from paper_1905_09554_gb300 import lbm  # noqa: E402

G0, TAU0 = -5.5, 0.9
RL, RV = inputs.COEXISTENCE[("shift", -5.5, 1.0)]


def neck_energy_np(rho):
    """Same objective as autograd.neck_energy, complex-safe numpy."""
    A = ((rho - RV) / (RL - RV)).sum(axis=(1, 2))
    R = np.sqrt(A / math.pi)
    return ((R - R.mean()) ** 2).mean()


def neck_energy_grad(rho):
    nz = rho.shape[0]
    A = ((rho - RV) / (RL - RV)).sum(axis=(1, 2))
    R = np.sqrt(A / math.pi)
    g = (2.0 / nz) * (R - R.mean()) / (2.0 * math.pi * R * (RL - RV))
    return np.broadcast_to(g[:, None, None], rho.shape).copy()


def small_case():
    return inputs.noisy_ligament_density(12, 12, 20, 3.0, 0.1, RL, RV, 1e-3, seed=31)


def oracle_J(rho0, G, tau, steps):
    p = o.Params(G=G, tau=tau, collision="srt")
    f = o.run(o.init_populations(rho0.astype(np.result_type(rho0, G, tau))), steps, p)
    return neck_energy_np(f.sum(0))


def gpu_grad(rho0, steps, every, storage="f64", G=G0, tau=TAU0):
    nz, ny, nx = rho0.shape
    with lbm.Lattice(nx, ny, nz, G=G, tau=tau, storage=storage) as L:
        L.adjoint_forward(rho0, steps, every)
        r, _ = L.moments()
        return L.adjoint_backward(neck_energy_grad(r))


def test_adjoint_matches_complex_step_of_the_reference():
    rho0 = small_case()
    steps = 30
    g_rho0, gG, gT = gpu_grad(rho0, steps, every=7)
    h = 1e-20
    rng = np.random.default_rng(5)
    for _ in range(2):
        v = rng.standard_normal(rho0.shape)
        cs = oracle_J(rho0 + 1j * h * v, G0, TAU0, steps).imag / h
        assert abs((g_rho0 * v).sum() - cs) <= 1e-9 * max(1.0, abs(cs)), (cs, (g_rho0 * v).sum())
    csG = oracle_J(rho0, G0 + 1j * h, TAU0, steps).imag / h
    csT = oracle_J(rho0, G0, TAU0 + 1j * h, steps).imag / h
    assert abs(gG - csG) <= 1e-9 * max(1e-6, abs(csG)), (gG, csG)
    assert abs(gT - csT) <= 1e-9 * max(1e-6, abs(csT)), (gT, csT)


def test_adjoint_matches_central_differences_of_the_gpu_forward():
    rho0 = small_case()
    steps = 25
    g_rho0, gG, gT = gpu_grad(rho0, steps, every=5)

    def J(r0=rho0, G=G0, tau=TAU0):
        nz, ny, nx = r0.shape
        with lbm.Lattice(nx, ny, nz, G=G, tau=tau, storage="f64") as L:
            L.set_density(r0)
            L.step(steps)
            r, _ = L.moments()
        return neck_energy_np(r)

    h = 1e-4
    v = np.random.default_rng(9).standard_normal(rho0.shape)
    fd = (J(r0=rho0 + h * v) - J(r0=rho0 - h * v)) / (2 * h)
    assert abs((g_rho0 * v).sum() - fd) <= 1e-6 * max(1e-8, abs(fd)) + 1e-12
    fdG = (J(G=G0 + h) - J(G=G0 - h)) / (2 * h)
    fdT = (J(tau=TAU0 + h) - J(tau=TAU0 - h)) / (2 * h)
    assert abs(gG - fdG) <= 1e-6 * max(1e-8, abs(fdG)) + 1e-12
    assert abs(gT - fdT) <= 1e-6 * max(1e-8, abs(fdT)) + 1e-12


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_conserved_objective_has_the_exact_gradient(storage, tol):
    """J = total mass at step T is conserved by the step, so dJ/drho0 = 1 in
    every cell and dJ/dG = dJ/dtau = 0, whatever the state: an exact answer
    that tests the whole reverse pass (collision, streaming and force
    adjoints and the parameter sums) with no reference to compare against."""
    rho0 = small_case()
    nz, ny, nx = rho0.shape
    with lbm.Lattice(nx, ny, nz, G=G0, tau=TAU0, storage=storage) as L:
        L.adjoint_forward(rho0, 40, 7)
        g, dG, dtau = L.adjoint_backward(np.ones_like(rho0))
    assert np.abs(g - 1.0).max() <= tol
    assert abs(dG) <= tol * rho0.size and abs(dtau) <= tol * rho0.size, (dG, dtau)


def test_checkpoint_interval_does_not_change_a_bit():
    rho0 = small_case()
    ref = gpu_grad(rho0, 24, every=24)
    for every in (1, 5, 7):
        got = gpu_grad(rho0, 24, every=every)
        assert np.array_equal(got[0], ref[0]) and got[1] == ref[1] and got[2] == ref[2], every


def test_fp32_adjoint_agrees_with_fp64():
    rho0 = small_case()
    g64 = gpu_grad(rho0, 30, every=6, storage="f64")
    g32 = gpu_grad(rho0, 30, every=6, storage="f32")
    scale = np.abs(g64[0]).max()
    assert np.abs(g32[0] - g64[0]).max() <= 2e-3 * scale
    assert abs(g32[1] - g64[1]) <= 2e-3 * abs(g64[1])
    assert abs(g32[2] - g64[2]) <= 2e-3 * abs(g64[2])


def test_adjoint_through_the_tensor_copy_kernel():
    """A context on the tensor-copy kernel (its segment recompute falls back
    to the pipelined kernel) gives the same gradients bit for bit."""
    rho0 = inputs.noisy_ligament_density(64, 32, 20, 5.0, 0.1, RL, RV, 1e-3, seed=33)
    out = []
    for kernel in (3, 5):
        with lbm.Lattice(64, 32, 20, G=G0, tau=TAU0, storage="f32", kernel=kernel, tile_y=16) as L:
            L.adjoint_forward(rho0, 12, 5)
            r, _ = L.moments()
            out.append(L.adjoint_backward(neck_energy_grad(r)))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1] and out[0][2] == out[1][2]


def test_torch_autograd_rollout():
    rho0_np = small_case()
    rho0 = torch.tensor(rho0_np, device="cuda", requires_grad=True)
    G = torch.tensor(G0, dtype=torch.float64, requires_grad=True)
    tau = torch.tensor(TAU0, dtype=torch.float64, requires_grad=True)
    J = lag.neck_energy(lag.rollout(rho0, G, tau, 30, every=7, storage="f64"), RL, RV)
    J.backward()
    assert abs(J.item() - oracle_J(rho0_np, G0, TAU0, 30)) <= 1e-12
    g_rho0, gG, gT = gpu_grad(rho0_np, 30, every=7)
    assert np.allclose(rho0.grad.cpu().numpy(), g_rho0, rtol=0, atol=1e-14 * np.abs(g_rho0).max())
    assert abs(G.grad.item() - gG) <= 1e-12 * abs(gG) and abs(tau.grad.item() - gT) <= 1e-12 * abs(gT)


def test_adjoint_refuses_mrt():
    with lbm.Lattice(8, 8, 8, collision="mrt", storage="f64") as L:
        with pytest.raises(lbm.LbmError, match="LBM_EUNSUPPORTED"):
            L.adjoint_forward(np.ones((8, 8, 8)), 4, 2)
