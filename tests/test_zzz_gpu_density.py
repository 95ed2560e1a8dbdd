"""Lattice.density() (lbm_moments with only rho requested, host output)
equals the rho of moments(), bit for bit."""

import numpy as np
import pytest

from paper_1905_09554_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CUDA device only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_09554_gb300 import lbm  # noqa: E402

RL, RV = inputs.COEXISTENCE[("shift", -5.5, 1.0)]


@pytest.mark.parametrize("storage", ["f32", "f16l"])
def test_density_alone_equals_moments_rho(storage):
    with lbm.Lattice(18, 14, 22, storage=storage) as L:
        L.init_ligament(4.0, 0.1, RL, RV)
        L.step(5)
        rho, _ = L.moments()
        assert np.array_equal(L.density(), rho)
