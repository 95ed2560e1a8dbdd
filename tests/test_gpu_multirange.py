"""The two-belt (multirange) force kernel (kernel 6) against the oracle's
two-belt step (oracle/multirange.py), and its equation of state on a flat
interface."""

import numpy as np
import pytest

from oracle import lbm_oracle as o
from oracle import multirange as mr
from paper_1905_09554_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CUDA device only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_09554_gb300 import calibration as cal  # noqa: E402
from paper_1905_09554_gb300 import lbm  # noqa: E402

RL, RV = inputs.COEXISTENCE[("shift", -5.5, 1.0)]


def gpu(rho, steps, storage, coll, tau, G1, G2, **kw):
    nz, ny, nx = rho.shape
    with lbm.Lattice(nx, ny, nz, G=G1, G2=G2, tau=tau, collision=coll, storage=storage, **kw) as L:
        assert L.kernel_config()["kernel"] == 6
        L.set_density(rho)
        L.step(steps)
        r, u = L.moments()
        return r, u


@pytest.mark.parametrize("coll", ["srt", "mrt"])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_two_belt_step_matches_the_oracle(coll, storage, tol):
    """Ragged 37 x 19 x 23 box (two tiles in x, the second partial; three in
    y), 20 steps, G1 = -7, G2 = +1.5 (the same G1 + G2 as the single-belt
    runs)."""
    rho = inputs.noisy_ligament_density(37, 19, 23, 5.0, 0.1, RL, RV, 1e-3, seed=11)
    p = o.Params(G=-7.0, tau=0.9, collision=coll)
    f = mr.run(o.init_populations(rho), 20, p, 1.5)
    r_ref, u_ref = mr.macroscopic(f, p, 1.5)
    r, u = gpu(rho, 20, storage, coll, 0.9, -7.0, 1.5, zchunk=7)
    assert np.abs(r - r_ref).max() <= tol
    assert np.abs(u - u_ref).max() <= tol


@pytest.mark.parametrize("shape", [(3, 2, 5), (1, 1, 4), (5, 9, 2)])
def test_two_belt_step_on_boxes_smaller_than_the_halo(shape):
    """Boxes with sides 1-5: the two-cell halo wraps several times."""
    nx, ny, nz = shape
    rho = inputs.random_density(nx, ny, nz, seed=5, lo=0.3, hi=1.9)
    p = o.Params(G=-4.0, tau=0.9, collision="srt")
    f = mr.run(o.init_populations(rho), 12, p, -1.0)
    r_ref, u_ref = mr.macroscopic(f, p, -1.0)
    r, u = gpu(rho, 12, "f64", "srt", 0.9, -4.0, -1.0)
    assert np.abs(r - r_ref).max() <= 1e-12
    assert np.abs(u - u_ref).max() <= 1e-12


@pytest.mark.parametrize("G1,G2", [(-5.5, 0.0), (-7.0, 1.5), (-4.5, -1.0)])
def test_flat_interface_pressure_balance_uses_g1_plus_g2(G1, G2):
    """Mechanical equilibrium of a flat interface: the bulk pressures
    P = rho cs2 + cs2 (G1 + G2) psi^2 / 2 of the two phases agree, for every
    split of G1 + G2 = -5.5 (MRT with unit rates)."""
    rl, rv, steps = cal.flat_coexistence(G1, 1.0, "mrt", G2=G2, rho_guess=(2.25, 0.06))
    pl, pv = cal.pressure(rl, G1, G2=G2), cal.pressure(rv, G1, G2=G2)
    assert rl > 1.5 and rv < 0.3, (rl, rv)
    assert abs(pl - pv) <= 1e-6 * abs(pl), (G1, G2, rl, rv, pl, pv, steps)  # measured <= 1.5e-9
    if G2 != 0:  # the first belt's strength alone does not balance
        assert abs(cal.pressure(rl, G1) - cal.pressure(rv, G1)) > 100 * abs(pl - pv)


def test_kernel_6_constraints():
    with pytest.raises(lbm.LbmError, match="LBM_EINVAL"):
        lbm.Lattice(8, 8, 8, storage="f16", G2=-1.0)
    with pytest.raises(lbm.LbmError, match="LBM_EINVAL"):
        lbm.Lattice(8, 8, 8, kernel=3, G2=-1.0)
    with pytest.raises(lbm.LbmError, match="LBM_EINVAL"):
        lbm.Lattice(8, 8, 8, kernel=6)
