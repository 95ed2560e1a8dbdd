"""The break-up driver (experiments.breakup_run) on a scripted fake lattice
with a known answer: a two-wave neck that closes linearly in time, the
break-up instant, satellite counting one capillary time after it, the
silhouettes / velocity snapshots and the pinch fit.  CPU only."""

import math

import numpy as np
import pytest

from paper_1905_09554_gb300 import experiments as ex

RL, RV = 2.0, 0.1
R0, NZ, TCAP = 10.0, 64, 100.0
T_PINCH = 850.0  # the neck radius reaches 0 at this step


class Scripted:
    """diag(): R(z) = R0 (1 - s(t) (1 + cos(2 pi 2 z / NZ)) / 2) with s rising
    linearly to 1 at T_PINCH (two necks, at z = 0 and NZ/2); slices with
    R < 0.5 hold no liquid.  After the pinch
    the two main drops plus one satellite between them remain, the satellite
    for `sat_life` steps."""

    def __init__(self, sat_life):
        self.t = 0
        self.sat_life = sat_life

    def step(self, n):
        self.t += n

    @property
    def time(self):
        return self.t

    def radius(self):
        z = np.arange(NZ)
        s = min(self.t / T_PINCH, 1.0)
        return R0 * (1.0 - s * 0.5 * (1.0 + np.cos(2 * math.pi * 2 * z / NZ)))

    def save(self, path):
        with open(path, "w") as fh:
            fh.write(str(self.t))

    def load(self, path):
        with open(path) as fh:
            self.t = int(fh.read())
        self.loaded_at = self.t

    def maxrho(self):
        R = self.radius()
        maxrho = np.where(R >= 0.5, RL, RV)
        if self.t >= T_PINCH:  # two drops around z = 16, 48 plus a satellite at z = 24
            maxrho = np.full(NZ, RV)
            maxrho[8:20] = RL
            maxrho[40:56] = RL
            if self.t < T_PINCH + self.sat_life:
                maxrho[23:26] = RL
        return maxrho

    def diag(self, rho_l, rho_v, raise_nonfinite=True):
        return {"status": 0, "maxrho_z": self.maxrho(), "area_z": math.pi * self.radius() ** 2}

    def density(self):
        rho = np.full((NZ, 4, 4), RV)
        rho[self.maxrho() == RL, :2, :] = RL  # liquid in half of each slice that holds some
        return rho

    def moments(self):
        rho = self.density()
        u = np.zeros((3, NZ, 4, 4))
        u[2, 5, 3, 3] = 0.7  # the fastest cell, in the vapour, at z = 5
        return rho, u


@pytest.mark.parametrize("sat_life,stable", [(40.0, 0), (500.0, 1)])
def test_breakup_run_on_a_scripted_ligament(sat_life, stable):
    L = Scripted(sat_life)
    res = ex.breakup_run(L, R0, TCAP, RL, RV, every=10, series=True, components=True)
    # break-up: first sample where a slice is dry, i.e. R < 0.5 at the neck
    # slices (z = 0, 32), s > 0.95 -> t > 807.5
    assert res["t_break"] is not None and 800.0 <= res["t_break"] <= 820.0
    assert res["T_break_over_tcap"] == pytest.approx(res["t_break"] / TCAP)
    # stops one t_cap after the first dry sample
    assert res["steps"] == pytest.approx(810 + 100, abs=10)
    assert res["drops_max"] == 3 and res["satellites_transient"] == 1
    assert res["satellites"] == stable
    # the final field read back: the same drops counted in 3D
    assert res["drops_3d"] == 2 + stable and res["satellites_3d"] == stable
    assert res["drop_volumes"][:2] == [16 * 8, 12 * 8]
    s = res["series"]
    assert set(s["silhouettes_R_over_R0"]) == {"7", "8"}  # t* = 9 is after the break-up
    assert len(s["silhouettes_R_over_R0"]["7"]) == NZ
    v = s["velocity_at_t_star"]["7"]
    assert v["v_max"] == pytest.approx(0.7 / (R0 / TCAP))
    assert v["v_max_vapour"] == pytest.approx(v["v_max"]) and v["v_max_liquid"] == 0.0
    assert v["z_of_max_from_neck_over_R0"] == pytest.approx(5 / R0)  # neck slice z = 0
    # the neck closes linearly: slope -R0 / T_PINCH per step = -1/8.5 R0 per t_cap
    fit = s["pinch_linear_fit"]
    assert fit["r2"] > 0.999 and fit["slope_R0_per_tcap"] == pytest.approx(-TCAP / T_PINCH, rel=1e-6)


def test_breakup_run_without_a_breakup_stops_at_the_limit():
    class Still(Scripted):
        def radius(self):
            return np.full(NZ, R0)

    res = ex.breakup_run(Still(0.0), R0, TCAP, RL, RV, every=50, max_tcap=3.0)
    assert res["t_break"] is None and res["T_break_over_tcap"] is None
    assert res["drops_max"] is None and res["satellites"] is None
    assert res["steps"] == 350  # the first sample past 3 t_cap ends the loop
    assert "drops_3d" not in ex.breakup_run(Still(0.0), R0, TCAP, RL, RV, every=50, max_tcap=1.0,
                                            components=True)


def test_breakup_run_resumes_from_its_checkpoint(tmp_path):
    """A run interrupted mid-way (here at step 530, after checkpoints every
    t_cap = 100 steps) and started again with the same checkpoint path
    returns exactly what the uninterrupted run returns."""
    want = ex.breakup_run(Scripted(40.0), R0, TCAP, RL, RV, every=10, series=True)

    class Crash(Exception):
        pass

    class Interrupted(Scripted):
        def step(self, n):
            if self.t >= 530:
                raise Crash()
            super().step(n)

    ck = str(tmp_path / "run.ckpt")
    with pytest.raises(Crash):
        ex.breakup_run(Interrupted(40.0), R0, TCAP, RL, RV, every=10, series=True, checkpoint=ck)
    resumed = Scripted(40.0)
    got = ex.breakup_run(resumed, R0, TCAP, RL, RV, every=10, series=True, checkpoint=ck)
    assert want["resumed_from_step"] == 0 and got["resumed_from_step"] == 500
    got["resumed_from_step"] = 0
    assert got == want
    assert resumed.loaded_at == 500  # the last checkpoint before the crash, not step 0


def test_breakup_run_resumes_after_a_crash_between_lattice_and_samples(tmp_path):
    """A crash after the lattice of a checkpoint is written but before its
    samples are committed: the resumed run starts from the previous complete
    checkpoint (lattice and samples of the same step) and returns what the
    uninterrupted run returns; no stale lattice file is left behind."""
    want = ex.breakup_run(Scripted(40.0), R0, TCAP, RL, RV, every=10, series=True)

    class Crash(Exception):
        pass

    class CrashInSave(Scripted):
        def save(self, path):
            super().save(path)
            if self.t >= 500:
                raise Crash()

    ck = str(tmp_path / "run.ckpt")
    with pytest.raises(Crash):
        ex.breakup_run(CrashInSave(40.0), R0, TCAP, RL, RV, every=10, series=True, checkpoint=ck)
    assert (tmp_path / "run.ckpt.t500").exists()  # written, never committed
    resumed = Scripted(40.0)
    got = ex.breakup_run(resumed, R0, TCAP, RL, RV, every=10, series=True, checkpoint=ck)
    assert resumed.loaded_at == 400
    assert got["resumed_from_step"] == 400
    got["resumed_from_step"] = 0
    assert got == want
    left = sorted(p.name for p in tmp_path.iterdir())
    assert left == ["run.ckpt.json", f"run.ckpt.t{max(int(n.split('.t')[-1]) for n in left if '.t' in n)}"]


def test_load_progress_refuses_a_lattice_of_another_step(tmp_path):
    import json

    ck = str(tmp_path / "run.ckpt")
    L = Scripted(0.0)
    L.t = 300
    ex._save_progress(L, ck, {"t": 300})
    with open(ck + ".json") as fh:
        state = json.load(fh)
    state["t"] = 400
    with open(ck + ".json", "w") as fh:
        json.dump(state, fh)
    with pytest.raises(RuntimeError):
        ex._load_progress(Scripted(0.0), ck)
