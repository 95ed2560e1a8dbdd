"""The OpenMP C reference step (oracle/c/lbm_ref.c) against the numpy
oracle: same definition, written independently (the MRT operator in C as
projections on the orthogonal moments, in numpy through the inverse
matrix), so they agree to rounding.  CPU only; skipped without a C
compiler."""

import shutil

import numpy as np
import pytest

from oracle import lbm_oracle as o
from paper_1905_09554_gb300 import inputs

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None and shutil.which("cc") is None,
                                reason="no C compiler")


@pytest.mark.parametrize("shape,G,tau", [((9, 7, 11), -5.5, 1.0), ((4, 5, 6), -4.0, 0.7), ((1, 1, 3), -5.5, 1.3)])
def test_c_reference_matches_the_numpy_oracle(shape, G, tau):
    from oracle import c_ref
    nx, ny, nz = shape
    rho = inputs.random_density(nx, ny, nz, seed=13, lo=0.2, hi=2.2)
    f0 = o.init_populations(rho)
    want = o.run(f0, 6, o.Params(G=G, tau=tau, collision="srt"))
    got = c_ref.run_srt(f0, 6, G, tau)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    assert c_ref.threads() >= 1


@pytest.mark.parametrize("rule,tau", [("paper", 0.8), ("random", 1.0)])
def test_c_reference_mrt_matches_the_numpy_oracle(rule, tau):
    from oracle import c_ref
    rho = inputs.random_density(6, 5, 7, seed=21, lo=0.2, hi=2.2)
    f0 = o.init_populations(rho)
    s = o.mrt_rates(tau) if rule == "paper" else np.random.default_rng(2).uniform(0.6, 1.8, 19)
    want = o.run(f0, 5, o.Params(G=-5.5, tau=tau, collision="mrt", s=s))
    got = c_ref.run_mrt(f0, 5, -5.5, s)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
