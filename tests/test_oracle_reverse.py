"""Pins of the reverse-mode FP64 reference (oracle/reverse.py): its forward
equals the numpy oracle's rollout, its gradients equal complex-step
derivatives of the numpy oracle (exact to rounding, no adjoint involved),
and a conserved objective has the exact gradient.  CPU only."""

import math

import numpy as np
import pytest

from oracle import lbm_oracle as o
from oracle import reverse as rv
from paper_1905_09554_gb300 import inputs

torch = pytest.importorskip("torch")

G0, TAU0 = -5.5, 0.9
RL, RV = inputs.COEXISTENCE[("shift", -5.5, 1.0)]


def small_case():
    return inputs.noisy_ligament_density(8, 8, 12, 2.0, 0.1, RL, RV, 1e-3, seed=31)


def oracle_J(rho0, G, tau, steps):
    p = o.Params(G=G, tau=tau, collision="srt")
    rho = o.run(o.init_populations(rho0.astype(np.result_type(rho0, G, tau))), steps, p).sum(0)
    A = ((rho - RV) / (RL - RV)).sum(axis=(1, 2))
    R = np.sqrt(A / math.pi)
    return ((R - R.mean()) ** 2).mean()


def test_forward_equals_the_numpy_oracle():
    rho0 = small_case()
    got = rv.rollout(torch.tensor(rho0), G0, TAU0, 15).numpy()
    want = o.run(o.init_populations(rho0), 15, o.Params(G=G0, tau=TAU0)).sum(0)
    assert np.abs(got - want).max() < 1e-13


def test_gradients_equal_complex_step_derivatives():
    rho0 = small_case()
    steps = 12
    J, g, gG, gT = rv.gradient(rho0, G0, TAU0, steps, "neck", RL, RV)
    assert abs(J - oracle_J(rho0, G0, TAU0, steps)) < 1e-14
    h = 1e-20
    rng = np.random.default_rng(3)
    for _ in range(2):
        v = rng.standard_normal(rho0.shape)
        cs = oracle_J(rho0 + 1j * h * v, G0, TAU0, steps).imag / h
        assert abs((g * v).sum() - cs) <= 1e-10 * max(1.0, abs(cs)), (cs, (g * v).sum())
    # one cell alone (the gradient field itself, not only its projections)
    e = np.zeros_like(rho0)
    e[5, 3, 4] = 1.0
    cs = oracle_J(rho0 + 1j * h * e, G0, TAU0, steps).imag / h
    assert abs(g[5, 3, 4] - cs) <= 1e-10 * max(1e-3, abs(cs))
    csG = oracle_J(rho0, G0 + 1j * h, TAU0, steps).imag / h
    csT = oracle_J(rho0, G0, TAU0 + 1j * h, steps).imag / h
    assert abs(gG - csG) <= 1e-10 * max(1e-6, abs(csG))
    assert abs(gT - csT) <= 1e-10 * max(1e-6, abs(csT))


def test_total_mass_has_the_exact_gradient():
    rho0 = small_case()
    _, g, gG, gT = rv.gradient(rho0, G0, TAU0, 10, "mass")
    assert np.abs(g - 1.0).max() < 1e-12 and abs(gG) < 1e-10 and abs(gT) < 1e-10


def test_density_misfit_gradient_equals_complex_step():
    """J = sum (rho(T) - target)^2 / 2 (the density L2 misfit)."""
    rho0 = small_case()
    target = inputs.noisy_ligament_density(8, 8, 12, 2.2, 0.05, RL, RV, 1e-3, seed=4)
    steps = 10

    def J_np(r0, G, tau):
        p = o.Params(G=G, tau=tau, collision="srt")
        rho = o.run(o.init_populations(r0.astype(np.result_type(r0, G, tau))), steps, p).sum(0)
        return 0.5 * ((rho - target) ** 2).sum()

    J, g, gG, gT = rv.gradient(rho0, G0, TAU0, steps, "misfit", target=target)
    assert abs(J - J_np(rho0, G0, TAU0)) <= 1e-12 * J
    h = 1e-20
    v = np.random.default_rng(8).standard_normal(rho0.shape)
    cs = J_np(rho0 + 1j * h * v, G0, TAU0).imag / h
    assert abs((g * v).sum() - cs) <= 1e-10 * max(1.0, abs(cs))
    assert abs(gG - J_np(rho0, G0 + 1j * h, TAU0).imag / h) <= 1e-10 * max(1e-6, abs(gG))
    assert abs(gT - J_np(rho0, G0, TAU0 + 1j * h).imag / h) <= 1e-10 * max(1e-6, abs(gT))
