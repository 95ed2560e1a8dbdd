"""The launch-shape autotuners on the GPU: lbm_tune (single lattice: kernel
variant, i.e. how the psi halo and the populations are staged, tile height
and z chunk) and lbm_batch_tune (batches: tile height and z chunk), and
their JSON caches.

Every step variant gives bit-identical states, so whatever shape the tuner
picks, the run it then makes must equal the register-staged kernel's bit for
bit; a cached pick is applied without timing."""

import numpy as np
import pytest

from paper_1905_09554_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CUDA device only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_09554_gb300 import lbm  # noqa: E402

RL, RV = inputs.COEXISTENCE[("shift", -5.5, 1.0)]


def _run(shape, storage, steps, **kw):
    nx, ny, nz = shape
    rho = inputs.noisy_ligament_density(nx, ny, nz, 5.0, 0.08, RL, RV, 1e-3, seed=21)
    with lbm.Lattice(nx, ny, nz, storage=storage, tau=0.8, **kw) as L:
        L.set_density(rho)
        L.step(steps)
        return L.get_populations()


@pytest.mark.parametrize("storage,shape", [("f32", (64, 40, 30)), ("f16l", (48, 36, 20)), ("f64", (33, 20, 12))])
def test_tuned_shape_steps_bit_identically(storage, shape):
    nx, ny, nz = shape
    with lbm.Lattice(nx, ny, nz, storage=storage, tau=0.8) as L:
        pick = L.tune(trial_steps=2)
        cfg = L.kernel_config()
        assert cfg["kernel"] == pick["kernel"] and cfg["tile_y"] == pick["tile_y"]
        assert pick["ms_per_step"] > 0 and not pick["cached"]
        rho = inputs.noisy_ligament_density(nx, ny, nz, 5.0, 0.08, RL, RV, 1e-3, seed=21)
        L.set_density(rho)
        L.step(6)
        f = L.get_populations()
    assert np.array_equal(f, _run(shape, storage, 6, kernel=1))


def test_lattice_tune_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    with lbm.Lattice(64, 32, 24, storage="f32") as L:
        first = L.tune(trial_steps=2, cache=path)
        assert not first["cached"]
    with lbm.Lattice(64, 32, 24, storage="f32") as L:
        again = L.tune(trial_steps=2, cache=path)
        assert again["cached"]
        assert {k: again[k] for k in ("kernel", "tile_y", "zchunk")} == \
            {k: first[k] for k in ("kernel", "tile_y", "zchunk")}
        cfg = L.kernel_config()
        assert (cfg["kernel"], cfg["tile_y"], cfg["zchunk"]) == (first["kernel"], first["tile_y"], first["zchunk"])
    with lbm.Lattice(64, 32, 26, storage="f32") as L:  # another box: tuned afresh
        assert not L.tune(trial_steps=2, cache=path)["cached"]


def test_set_kernel_config_refuses_bad_shapes_and_keeps_the_old_one():
    with lbm.Lattice(40, 16, 12, storage="f32") as L:
        L.set_kernel_config(3, 8, 4)
        before = L.kernel_config()
        assert (before["kernel"], before["tile_y"], before["zchunk"]) == (3, 8, 4)
        for bad in ((7, 8, 0), (3, 12, 0), (6, 8, 0), (5, 16, 0)):  # 16-bit only; tile; two-belt; nx % 32
            with pytest.raises(lbm.LbmError, match="LBM_EINVAL"):
                L.set_kernel_config(*bad)
            assert L.kernel_config() == before


def test_batch_tune_cache_round_trip(tmp_path):
    path = str(tmp_path / "batch_tune.json")
    dims = [(32, 32, 40), (48, 48, 36), (32, 32, 70)]
    with lbm.Batch(dims, storage="f32", tune_cache=path) as B:
        first = B.config()
    data = lbm._read_tune_cache(path)
    assert len(data) == 1
    entry = next(iter(data.values()))
    assert (entry["tile_y"], entry["zchunk"]) == (first["tile_y"], first["zchunk"])
    with lbm.Batch(dims, storage="f32", tune_cache=path) as B:
        again = B.config()
    assert (again["tile_y"], again["zchunk"]) == (first["tile_y"], first["zchunk"])
    assert lbm._read_tune_cache(path) == data  # used, not retuned
