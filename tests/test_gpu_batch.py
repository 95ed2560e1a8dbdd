"""Batched form: many independent periodic ligament boxes of uneven size
advanced by one kernel launch per step (pairs of steps replayed from a CUDA
graph).  Every box must evolve exactly as the same box alone: the batched
kernel runs the same per-cell arithmetic, so the states are bit-identical."""

import math

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
DIMS = [(32, 32, 50), (20, 17, 33), (48, 48, 75), (33, 40, 9), (5, 7, 3), (64, 64, 101)]


def box_density(k, nx, ny, nz):
    R0 = max(1.5, min(nx, ny) / 4.0)
    return inputs.noisy_ligament_density(nx, ny, nz, R0, 0.03, RL, RV, 1e-3, seed=20 + k)


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("coll", ["srt", "mrt"])
def test_batch_boxes_match_single_boxes_bit_for_bit(storage, coll):
    steps = [3, 2, 1, 4]  # odd and even counts exercise the graph and plain launches
    with lbm.Batch(DIMS, G=G, tau=0.9, collision=coll, storage=storage) as B:
        for k, v in enumerate(B.boxes):
            v.set_density(box_density(k, *DIMS[k]))
        for s in steps:
            B.step(s)
        got = [v.get_populations() for v in B.boxes]
        assert all(v.time == sum(steps) for v in B.boxes)
    for k, (nx, ny, nz) in enumerate(DIMS):
        with lbm.Lattice(nx, ny, nz, G=G, tau=0.9, collision=coll, storage=storage) as L:
            L.set_density(box_density(k, nx, ny, nz))
            L.step(sum(steps))
            want = L.get_populations()
        assert np.array_equal(got[k], want), (k, DIMS[k])


def test_batch_box_matches_the_reference():
    with lbm.Batch(DIMS[:3], G=G, tau=1.0, storage="f64") as B:
        for k, v in enumerate(B.boxes):
            v.set_density(box_density(k, *DIMS[k]))
        B.step(40)
        r, u = B.boxes[1].moments()
    p = o.Params(G=G, tau=1.0)
    r_ref, u_ref = o.macroscopic(o.run(o.init_populations(box_density(1, *DIMS[1])), 40, p), p)
    assert np.abs(r - r_ref).max() <= 1e-12
    assert np.abs(u - u_ref).max() <= 1e-12


def test_autotune_then_run_is_still_exact():
    with lbm.Batch(DIMS, G=G, tau=1.0, storage="f32") as B:
        best = B.tune(trial_steps=2)
        assert best["tile_y"] in (4, 8, 16) and best["zchunk"] in (8, 16, 24, 32, 48, 64)
        assert best["ms_per_step"] > 0
        cfg = B.config()
        assert (cfg["tile_y"], cfg["zchunk"]) == (best["tile_y"], best["zchunk"])
        assert cfg["cells"] == sum(a * b * c for a, b, c in DIMS)
        for k, v in enumerate(B.boxes):
            v.set_density(box_density(k, *DIMS[k]))
        B.step(6)
        got = B.boxes[2].get_populations()
    with lbm.Lattice(*DIMS[2], G=G, tau=1.0, storage="f32") as L:
        L.set_density(box_density(2, *DIMS[2]))
        L.step(6)
        assert np.array_equal(got, L.get_populations())


def test_box_views_cannot_be_stepped_or_freed_alone():
    with lbm.Batch(DIMS[:2], storage="f32") as B:
        with pytest.raises(lbm.LbmError, match="LBM_EINVAL"):
            B.boxes[0].step(1)
        assert lbm.lbm_step(B.boxes[0].ctx, 1) == lbm.LBM_EINVAL
        lbm.lbm_destroy(B.boxes[0].ctx)  # ignored: owned by the batch
        B.step(2)
        assert B.boxes[0].time == 2


def test_batch_rejects_16_bit_storage():
    with pytest.raises(lbm.LbmError, match="LBM_EINVAL"):
        lbm.Batch(DIMS[:2], storage="f16")
