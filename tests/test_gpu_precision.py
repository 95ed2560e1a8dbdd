"""Low-precision population storage (FP16 / BF16 deviations from the rest
equilibrium at rho_ref, scaled), float arithmetic; and the local-reference
formats, where rho_ref is a per-cell float field R(x): the cell's density
when the populations are set, and the density before the step after each
step.

* Encoding: set/get populations round-trips through exactly the documented
  format d = (f - w rho_ref) * scale rounded to the 16-bit type.
* One step: the GPU result equals the FP64 reference step applied to the
  decoded input, up to one unit in the last place of the stored 16-bit
  deviation.
* Many steps: the error against the FP64 reference after 200 steps of the
  small ligament stays within the bound this file states per format.
"""

import numpy as np
import pytest

from oracle import lbm_oracle as o
from paper_1905_09554_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CUDA device only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_09554_gb300 import lbm  # noqa: E402

G = -5.5
RL, RV = inputs.COEXISTENCE[("shift", G, 1.0)]
EPS = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8, "f16l": 2.0 ** -11, "bf16l": 2.0 ** -8}  # unit roundoff
BASE = {"f16": "f16", "bf16": "bf16", "f16l": "f16", "bf16l": "bf16"}  # 16-bit type of the format


def lib_weights():
    return lbm.lbm_velocities()[1]


def perm():
    c, _ = lbm.lbm_velocities()
    ref = {tuple(v): i for i, v in enumerate(o.C)}
    return np.array([ref[tuple(v)] for v in c])


def to_ref(f_lib):
    out = np.empty_like(f_lib)
    out[perm()] = f_lib
    return out


def to_lib(f_ref):
    return f_ref[perm()]


def bf16_round(x32):
    b = x32.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32)


def emulate(f_lib, fmt, rho_ref, scale):
    """Host emulation of the storage round trip (float32 arithmetic);
    rho_ref is a scalar or a per-cell array."""
    w = lib_weights().astype(np.float32).reshape((19,) + (1,) * (f_lib.ndim - 1))
    R = np.asarray(rho_ref, dtype=np.float32)
    d = (f_lib.astype(np.float32) - w * R) * np.float32(scale)
    dq = d.astype(np.float16).astype(np.float32) if BASE[fmt] == "f16" else bf16_round(d)
    return (w * R + dq * np.float32(1.0 / scale)).astype(np.float64), d


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("rho_ref,scale", [(1.0, 1.0), (1.2, 8.0)])
def test_storage_round_trip(fmt, rho_ref, scale):
    rho = inputs.ligament_density(24, 16, 20, 4.0, 0.1, RL, RV)
    f = to_lib(o.init_populations(rho)) * (1 + 0.01 * inputs.gaussian(19 * rho.size, 3).reshape((19,) + rho.shape))
    with lbm.Lattice(24, 16, 20, storage=fmt, rho_ref=rho_ref, dev_scale=scale) as L:
        L.set_populations(f)
        got = L.get_populations()
    want, d = emulate(f, fmt, rho_ref, scale)
    # The device may fuse the subtraction and the scaling (one rounding
    # fewer than the host emulation), which can move a value that sits next
    # to a rounding boundary by one stored unit; nothing else may differ.
    one_unit = 2 * EPS[fmt] * np.abs(d) / scale + 1e-7
    assert (np.abs(got - want) <= one_unit).all()
    assert np.mean(got == want) > 0.99
    assert np.abs(got - f).max() <= EPS[fmt] * np.abs(d).max() / scale + 1e-6


@pytest.mark.parametrize("fmt", ["f16l", "bf16l"])
@pytest.mark.parametrize("scale", [1.0, 8.0])
def test_local_storage_round_trip(fmt, scale):
    """The reference of each cell is the float32 sum of its populations."""
    rho = inputs.ligament_density(24, 16, 20, 4.0, 0.1, RL, RV)
    f = to_lib(o.init_populations(rho)) * (1 + 0.01 * inputs.gaussian(19 * rho.size, 3).reshape((19,) + rho.shape))
    with lbm.Lattice(24, 16, 20, storage=fmt, rho_ref=123.0, dev_scale=scale) as L:
        L.set_populations(f)
        got = L.get_populations()
        got_rho = L.moments()[0]
    R = f.sum(axis=0).astype(np.float32)
    want, d = emulate(f, fmt, R, scale)
    # one stored unit: relative 2u for normal values, 2^-24 for FP16
    # subnormals (tiny deviations of cells near the rest state)
    sub = 2.0 ** -24 if BASE[fmt] == "f16" else 0.0
    one_unit = (2 * EPS[fmt] * np.abs(d) + sub) / scale + 4e-7 * R
    assert (np.abs(got - want) <= one_unit).all()
    assert np.mean(got == want) > 0.95
    # the deviations are only the 1% noise: the stored error is tiny
    assert np.abs(got - f).max() <= (2 * EPS[fmt] * np.abs(d).max() + sub) / scale + 4e-7 * R.max()
    # moments decode with the same per-cell reference (rho summed in float)
    assert np.abs(got_rho - got.sum(axis=0)).max() <= 5e-6 * RL


@pytest.mark.parametrize("fmt", ["f16l", "bf16l"])
def test_local_rest_state_is_exact(fmt):
    """Populations at rest equilibrium store (up to the float rounding of
    w_a rho) zero deviations: decoding gives w_a R, R the float32 density."""
    rho = inputs.ligament_density(20, 12, 16, 3.0, 0.1, RL, RV)
    with lbm.Lattice(20, 12, 16, storage=fmt) as L:
        L.set_density(rho)
        got = L.get_populations()
    w = lib_weights().astype(np.float32).reshape((19, 1, 1, 1))
    want = (w * rho.astype(np.float32)).astype(np.float64)
    assert (np.abs(got - want) <= 2.5e-7 * want).all()


@pytest.mark.parametrize("fmt", ["f16", "bf16", "f16l", "bf16l"])
@pytest.mark.parametrize("coll", ["srt", "mrt"])
def test_one_step_within_one_stored_ulp(fmt, coll):
    rho = inputs.noisy_ligament_density(33, 18, 20, 5.0, 0.1, RL, RV, 1e-3, seed=8)
    with lbm.Lattice(33, 18, 20, G=G, tau=0.9, collision=coll, storage=fmt, rho_ref=1.0) as L:
        L.set_density(rho)
        f_in = L.get_populations()
        L.step(1)
        got = L.get_populations()
    h = to_lib(o.step(to_ref(f_in), o.Params(G=G, tau=0.9, collision=coll)))
    w = lib_weights().reshape((19, 1, 1, 1))
    # deviations of the destination cell: from rho_ref = 1, or for the local
    # formats from that cell's density before the step
    R = f_in.sum(axis=0) if fmt.endswith("l") else 1.0
    ulp = 2 * EPS[fmt] * np.abs(h - w * R)
    assert (np.abs(got - h) <= ulp + 2e-6).all()


# Bound on max |rho - rho_FP64| after 200 steps of the 32x32x64 ligament
# (rho_ref = 1, scale 1): the stored deviation is rounded every step with
# relative error u (2^-11 FP16, 2^-8 BF16) and |d| <= 0.45 w, so rho drifts
# by a few u per step.  Measured on GB300: FP16 2.2e-3, BF16 1.9e-1 (BF16's
# 8-bit significand is too coarse for this two-phase state); the bounds are
# ~2.5x those values and catch a broken codec, not a precision claim.  The
# local-reference formats store only the non-equilibrium part and the
# density change of one step (|d| ~ 1e-2 w at the interface), so their
# rounding error per step is smaller by that ratio.
BOUND_200 = {"f16": 5e-3, "bf16": 0.5, "f16l": 1e-3, "bf16l": 5e-2}


@pytest.mark.parametrize("fmt", ["f16", "bf16", "f16l", "bf16l", "f32"])
def test_error_after_200_steps_vs_fp64(fmt):
    rho0 = inputs.ligament_density(32, 32, 64, 8.0, 0.05, RL, RV)
    p = o.Params(G=G, tau=1.0, collision="srt")
    r_ref, u_ref = o.macroscopic(o.run(o.init_populations(rho0), 200, p), p)
    with lbm.Lattice(32, 32, 64, G=G, tau=1.0, storage=fmt, rho_ref=1.0) as L:
        L.set_density(rho0)
        L.step(200)
        r, u = L.moments()
    err_r, err_u = np.abs(r - r_ref).max(), np.abs(u - u_ref).max()
    print(f"{fmt}: max|drho| = {err_r:.3e}, max|du| = {err_u:.3e}")
    bound = BOUND_200.get(fmt, 2e-5)
    assert err_r <= bound
