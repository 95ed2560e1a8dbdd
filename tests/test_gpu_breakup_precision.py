"""FP32 against FP64 storage over a whole break-up run (Sec. 4: break-up
time of the perturbed ligament), on the GPU.

The ligament R0 = 16, kR0 = 0.7 (box 64 x 64 x 144, one wavelength along z,
5% cosine perturbation, G = -5.5) runs to pinch-off with FP64 and with FP32
populations, for SRT (tau = 1) and MRT with Guo forcing (shear moments at
1/tau = 1.25, bulk and ghost moments at 1).  Diagnostics are sampled every 5
steps (a capillary time is ~300 steps); the break-up time is the first
sample with a slice free of liquid, interpolated linearly between samples.

Bars: the FP32 break-up time within 1% of the FP64 one, and the FP32
density within 2e-5 (max abs) of the FP64 density after 200 steps.
"""

import numpy as np
import pytest

from paper_1905_09554_gb300 import diagnostics as dg
from paper_1905_09554_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CUDA device only
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1905_09554_gb300 import lbm  # noqa: E402

R0, KR0, EPS, EVERY, MAX_STEPS = 16.0, 0.7, 0.05, 5, 20000


def _rates(coll, tau):
    if coll == "srt":
        return None
    s = [1.0] * 19
    for k in (9, 11, 13, 14, 15):  # 3pxx, pww, pxy, pyz, pxz
        s[k] = 1.0 / tau
    return s


def _run(storage, coll, tau):
    forcing = "shift" if coll == "srt" else "guo"
    rl, rv = inputs.COEXISTENCE[(forcing, -5.5, 1.0)]
    nx, ny, nz = inputs.ligament_box(R0, KR0)
    with lbm.Lattice(nx, ny, nz, G=-5.5, tau=tau, collision=coll, rates=_rates(coll, tau),
                     storage=storage) as L:
        L.init_ligament(R0, EPS, rl, rv)
        L.step(200)
        rho200 = L.density()
        ts, mins = [], []
        t = 200
        while t <= MAX_STEPS:
            d = L.diag(rl, rv)
            ts.append(t)
            mins.append(float(d["maxrho_z"].min()))
            if mins[-1] < 0.5 * (rl + rv):
                break
            L.step(EVERY)
            t += EVERY
    return rho200, dg.breakup_time(ts, mins, rl, rv)


@pytest.mark.parametrize("coll,tau", [("srt", 1.0), ("mrt", 0.8)])
def test_fp32_breakup_time_within_one_percent_of_fp64(coll, tau):
    rho64, tb64 = _run("f64", coll, tau)
    rho32, tb32 = _run("f32", coll, tau)
    assert tb64 is not None and tb32 is not None, "no break-up within the run"
    rel = abs(tb32 - tb64) / tb64
    err200 = float(np.abs(rho32 - rho64).max())
    print(f"{coll} tau={tau}: T_break FP64 {tb64:.2f}, FP32 {tb32:.2f} steps (rel {rel:.2e}); "
          f"max|rho32 - rho64| at step 200 = {err200:.2e}")
    assert rel <= 0.01
    assert err200 <= 2e-5
