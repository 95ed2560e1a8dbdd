"""The OpenMP C reference step (oracle/c/lbm_ref.c) against the numpy
reference: same definition, written independently, so they agree to
rounding.  CPU only; skipped without a C compiler."""

import shutil

import numpy as np
import pytest

from oracle import lbm_oracle as o
from paper_1905_09554_gb300 import inputs

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None and shutil.which("cc") is None,
                                reason="no C compiler")


@pytest.mark.parametrize("shape,G,tau", [((9, 7, 11), -5.5, 1.0), ((4, 5, 6), -4.0, 0.7), ((1, 1, 3), -5.5, 1.3)])
def test_c_reference_matches_the_numpy_reference(shape, G, tau):
    from oracle import c_ref
    nx, ny, nz = shape
    rho = inputs.random_density(nx, ny, nz, seed=13, lo=0.2, hi=2.2)
    f0 = o.init_populations(rho)
    want = o.run(f0, 6, o.Params(G=G, tau=tau, collision="srt"))
    got = c_ref.run_srt(f0, 6, G, tau)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    assert c_ref.threads() >= 1
