"""The paper's break-up run (Secs. 3-4) as a driver over a lattice: step to
the pinch-off while sampling the diagnostics, count the drops for a
capillary time after it, and optionally record the series behind Figs. 5-7.

Works with any object that has the `Lattice` methods it uses (`diag`,
`step`, `moments`); the arithmetic of the step is the library's.  Host-side
analysis only (numpy), built on `diagnostics`.
"""

from __future__ import annotations

import numpy as np

from . import diagnostics as dg

SNAPSHOT_T_STAR = (7, 8, 9)  # silhouettes and velocity (Figs. 5b and 7)


def pinch_linear_fit(t_star, neck_over_R0, hi=0.3, lo=0.05, min_points=3):
    """Least-squares line of R_min/R0 against t* over the samples with
    lo <= R_min/R0 <= hi (the final pinch, Fig. 6): slope, points, r^2."""
    tt = np.asarray(t_star, dtype=float)
    nk = np.asarray(neck_over_R0, dtype=float)
    sel = (nk <= hi) & (nk >= lo)
    if sel.sum() < min_points:
        return None
    sl, ic = np.polyfit(tt[sel], nk[sel], 1)
    fit = sl * tt[sel] + ic
    ss = float(((nk[sel] - nk[sel].mean()) ** 2).sum())
    return {"slope_R0_per_tcap": float(sl), "points": int(sel.sum()),
            "r2": 1.0 - float(((nk[sel] - fit) ** 2).sum()) / ss if ss > 0 else 1.0}


def velocity_snapshot(rho, u, rho_l, rho_v, R0, tcap, Rz):
    """Where v* = |u_b| / (R0 / t_cap) peaks (Fig. 7): overall, in the vapour
    (rho below the mid density) and in the liquid, and the distance in z of
    the peak from the neck slice, in units of R0."""
    nz = rho.shape[0]
    vs = np.sqrt((u ** 2).sum(axis=0)) / (R0 / tcap)
    vap = rho < 0.5 * (rho_l + rho_v)
    zmax = int(np.unravel_index(int(np.argmax(vs)), vs.shape)[0])
    zneck = int(np.argmin(Rz))
    dz = min(abs(zmax - zneck), nz - abs(zmax - zneck))
    return {"v_max": float(vs.max()),
            "v_max_vapour": float(vs[vap].max()) if vap.any() else None,
            "v_max_liquid": float(vs[~vap].max()) if (~vap).any() else None,
            "z_of_max_from_neck_over_R0": dz / R0}


def _lattice_file(path, t):
    return f"{path}.t{int(t)}"


def _save_progress(L, path, state):
    """Checkpoint of the run: the lattice at step state["t"] in its own file
    (path + ".t<step>"), then the sampled state, naming that file, in
    path + ".json" (written to a temporary name and renamed), then the older
    lattice files are removed.  The json is the commit point: a crash before
    its rename leaves the previous json and the lattice file it names intact,
    so a resumed run never pairs a lattice with samples of another step."""
    import glob
    import json
    import os

    lat = _lattice_file(path, state["t"])
    L.save(lat)
    tmp = f"{path}.json.tmp"
    with open(tmp, "w") as fh:
        json.dump(dict(state, lattice=os.path.basename(lat)), fh)
    os.replace(tmp, path + ".json")
    for old in glob.glob(glob.escape(path) + ".t[0-9]*"):
        if old != lat and old[len(path) + 2:].isdigit():
            os.remove(old)


def _load_progress(L, path):
    """The sampled state saved with the last complete checkpoint at `path`
    (after restoring the lattice from the file it names), or None if there
    is none.  Raises if the restored lattice is not at the state's step."""
    import json
    import os

    if not os.path.exists(path + ".json"):
        return None
    with open(path + ".json") as fh:
        state = json.load(fh)
    lat = os.path.join(os.path.dirname(path), state.get("lattice", ""))
    if not state.get("lattice") or not os.path.exists(lat):
        return None
    L.load(lat)
    if L.time != state["t"]:
        raise RuntimeError(f"checkpoint {lat} holds step {L.time}, its samples end at step {state['t']}")
    return state


def breakup_run(L, R0, tcap, rho_l, rho_v, every, series=False, max_tcap=30.0, after_tcap=1.0, n_waves=2,
                components=False, checkpoint=None, checkpoint_every=None):
    """Step `L` (already initialised) in strides of `every` steps, sampling
    `L.diag` before each stride, until some z slice holds no liquid (the
    break-up), then for `after_tcap` capillary times more while counting the
    drops on the axis.  Stops early on a non-finite state or after
    `max_tcap` capillary times.

    Returns a dict: steps, t_break (steps, interpolated) and
    T_break_over_tcap (None if no break-up), drops_max / drops_final and the
    satellites (drops beyond the n_waves main ones at the end / at most), and
    with `series` the neck-radius and mode-amplitude series, the silhouettes
    and velocity snapshots at t* = 7, 8, 9 (first sample past each) and the
    linear fit of the final pinch.  With `components` (and a break-up) the
    final density field is read back and its drops counted in 3D
    (`diagnostics.drop_components`): drops_3d, their cell counts, and the
    satellites_3d beyond the n_waves main drops.

    With `checkpoint` (a file path) the run saves the lattice (`L.save`, to
    path + ".t<step>") and its sampled series (path + ".json") every
    `checkpoint_every` steps (default: one capillary time) and, if a complete
    checkpoint exists when it starts, resumes from it: an interrupted run continued this way returns what
    the uninterrupted one would (apart from resumed_from_step, the step it
    started at: 0 for a fresh run)."""
    ts, mins, drops = [], [], []
    necks, amps, sil, vel = [], [], {}, {}
    t, broke_at, status = 0, None, 0
    if checkpoint is not None:
        every_ck = int(checkpoint_every or max(every, round(tcap)))
        state = _load_progress(L, checkpoint)
        if state is not None:
            t, broke_at = state["t"], state["broke_at"]
            ts, mins, drops = state["ts"], state["mins"], state["drops"]
            necks, amps = state["necks"], state["amps"]
            sil = {int(k): v for k, v in state["sil"].items()}
            vel = {int(k): v for k, v in state["vel"].items()}
        next_ck = t + every_ck
    t_start = t
    while t <= max_tcap * tcap:
        if checkpoint is not None and t >= next_ck:
            _save_progress(L, checkpoint, {"t": t, "broke_at": broke_at, "ts": ts, "mins": mins, "drops": drops,
                                           "necks": necks, "amps": amps, "sil": sil, "vel": vel})
            next_ck = t + every_ck
        d = L.diag(rho_l, rho_v, raise_nonfinite=False)
        status = d["status"]
        if status != 0:
            break
        if broke_at is None:
            ts.append(t)
            mins.append(float(d["maxrho_z"].min()))
            if series:
                necks.append(dg.neck_radius(d["area_z"]) / R0)
                amps.append(dg.mode_amplitude(d["area_z"], n_waves=n_waves))
                for ts_star in SNAPSHOT_T_STAR:
                    if ts_star not in sil and t >= ts_star * tcap:
                        Rz = dg.equivalent_radius(d["area_z"])
                        sil[ts_star] = [round(float(v) / R0, 4) for v in Rz]
                        rho, u = L.moments()
                        vel[ts_star] = velocity_snapshot(rho, u, rho_l, rho_v, R0, tcap, Rz)
                        del rho, u
            if mins[-1] < 0.5 * (rho_l + rho_v):
                broke_at = t
        if broke_at is not None:
            drops.append(dg.count_drops(d["maxrho_z"], rho_l, rho_v))
            if t >= broke_at + after_tcap * tcap:
                break
        L.step(every)
        t += every
    tb = dg.breakup_time(ts, mins, rho_l, rho_v)
    out = {"steps": t, "status": status, "t_break": tb, "resumed_from_step": t_start,
           "T_break_over_tcap": tb / tcap if tb is not None else None,
           "drops_max": max(drops) if drops else None, "drops_final": drops[-1] if drops else None,
           "satellites": max(0, drops[-1] - n_waves) if drops else None,
           "satellites_transient": max(0, max(drops) - n_waves) if drops else None}
    if components and broke_at is not None and status == 0:
        rho = L.density()
        vols = dg.drop_components(rho, rho_l, rho_v)
        del rho
        out.update({"drops_3d": len(vols), "drop_volumes": vols, "satellites_3d": max(0, len(vols) - n_waves)})
    if series and ts:
        tt = np.asarray(ts[:len(necks)], dtype=float) / tcap
        a0 = amps[0] if amps and amps[0] != 0 else 1.0
        out["series"] = {"t_star": [round(float(v), 4) for v in tt],
                         "neck_over_R0": [round(float(v), 4) for v in necks],
                         "mode_amplitude_over_initial": [round(float(v) / a0, 4) for v in amps],
                         "silhouettes_R_over_R0": {str(k): v for k, v in sil.items()},
                         "velocity_at_t_star": {str(k): v for k, v in vel.items()},
                         "pinch_linear_fit": pinch_linear_fit(tt, necks)}
    return out
