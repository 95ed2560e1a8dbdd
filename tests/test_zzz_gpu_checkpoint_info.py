"""lbm_checkpoint_info on files written by lbm_save: the header read on the
host alone matches the context that wrote it, and the checksum verifies."""

import pytest

from paper_1905_09554_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CUDA device only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_09554_gb300 import lbm  # noqa: E402

RL, RV = inputs.COEXISTENCE[("shift", -5.5, 1.0)]


@pytest.mark.parametrize("storage,collision", [("f32", "srt"), ("bf16l", "mrt")])
def test_info_of_a_saved_state(tmp_path, storage, collision):
    path = str(tmp_path / "state.ckpt")
    with lbm.Lattice(20, 12, 28, G=-5.3, tau=0.8, collision=collision, storage=storage) as L:
        L.init_ligament(4.0, 0.1, RL, RV)
        L.step(9)
        L.save(path)
    info = lbm.checkpoint_info(path)
    assert info["dims"] == (20, 12, 28) and info["t"] == 9
    assert info["storage"] == lbm.STORAGE[storage] and info["collision"] == lbm.COLLISION[collision]
    assert info["G"] == -5.3 and info["tau"] == 0.8
