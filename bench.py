#!/usr/bin/env python
"""Benchmark of the D3Q19 Shan-Chen lattice Boltzmann step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (default): the sharp-interface ligament R0 = 64, kR0 = 0.7 in a
256 x 256 x 575 periodic box (37.7 M cells), G = -5.5, SRT with velocity shift
at tau = 1, FP32 populations, 5% cosine perturbation.  A step is one fused
step-kernel launch over the whole box; inputs (2 x 2.86 GB population copies)
are far larger than L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  `value` is MLUPS (million lattice updates per
second) over all ranks, device-timed with CUDA events; `e2e` is the same
metric through the C ABI with host buffers (initial density uploaded from
pinned host memory, diagnostics read back every 50 steps, final density read
back); `roofline` relates the step kernel's algorithmic bytes to the measured
HBM copy bandwidth; `cpu_baseline` times the FP64 reference implementation on
a bounded slab of the same workload on the host cores.

With N > 1 (torchrun) every rank advances its own replica of the ligament
(weak scaling; the step has no data-path collective).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q19 SC-LBM MLUPS & % HBM peak; FP32/FP16 & batched vs FP64 at stated error"
BYTES_PER_POP = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2, "f16l": 2, "bf16l": 2}
# local-reference formats also read and write a float reference density per cell
EXTRA_BYTES_PER_CELL = {"f16l": 8, "bf16l": 8}
FALLBACK_HBM_GBS = 6800.0
KERNEL_NAMES = {1: "sc_step_kernel", 2: "sc_step_async_kernel", 3: "sc_step_pipe_kernel", 4: "sc_step_bulk_kernel",
                5: "sc_step_tma_kernel", 6: "sc_step_mr_kernel", 7: "sc_step_pair16_kernel"}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--collision", choices=["srt", "mrt"], default="srt")
    ap.add_argument("--storage", choices=list(BYTES_PER_POP), default="f32")
    ap.add_argument("--R0", type=float, default=64.0)
    ap.add_argument("--kR0", type=float, default=0.7)
    ap.add_argument("--tau", type=float, default=1.0)
    ap.add_argument("--G2", type=float, default=0.0,
                    help="single form: second belt of the two-belt force (kernel 6); the first belt is then "
                         "-5.5 - G2, so the bulk EoS stays that of G = -5.5")
    ap.add_argument("--mrt-rule", choices=["shear", "paper"], default="shear",
                    help="MRT rates: shear moments at 1/tau (shear) or also the energy moment (paper)")
    ap.add_argument("--zchunk", type=int, default=0)
    ap.add_argument("--tile-y", type=int, default=0)
    ap.add_argument("--kernel", type=int, default=0, help="0 auto, 1 register-staged, 2 cp.async-staged, 3 pipelined, 4 bulk-copy, "
                         "5 tensor-copy, 7 paired 16-bit")
    ap.add_argument("--e2e-steps", type=int, default=1000)
    ap.add_argument("--e2e-diag-every", type=int, default=50,
                    help="e2e: steps between diagnostics read back to the host (the paper's break-up runs "
                         "sample every t_cap/40, 63 steps for the R0 = 64 ligament)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="single form: skip the FP64 / 16-bit / batched / adjoint record beside the headline")
    ap.add_argument("--form", choices=["single", "batched", "adjoint", "precision", "paper", "calibrate", "multirange"],
                    default="single",
                    help="single: the sharp-interface ligament; batched: 64 uneven ligaments in one launch per "
                         "step; adjoint: gradients of the neck energy through 500 steps; precision: FP32/FP16/BF16 "
                         "storage against FP64; paper: the break-up experiment at the paper's parameters; "
                         "calibrate: the Sec. 3 Laplace / flat-interface / Oh calibration against Tables 1-2")
    ap.add_argument("--series", action="store_true",
                    help="paper form: also report the neck-radius and perturbation time series, the interface "
                         "silhouettes at t* = 7, 8, 9 and the linearity of the final pinch")
    ap.add_argument("--checkpoint-dir", default=None,
                    help="paper form: checkpoint each run there every capillary time and resume an interrupted "
                         "run from its checkpoint (a file holds one population copy: 61 GB at R0 = 98; the "
                         "previous file is removed only after the next one is complete)")
    ap.add_argument("--components", action="store_true",
                    help="paper form: also count the drops of the final state in 3D (connected components of "
                         "the liquid; reads the density field back to the host)")
    ap.add_argument("--tau0", type=float, default=0.75, help="calibrate form: starting SRT relaxation time")
    ap.add_argument("--cal-tol", type=float, default=0.01,
                    help="calibrate form: stop when two consecutive sigma agree to this fraction")
    ap.add_argument("--radii", default="14,28,42",
                    help="paper form: ligament radii of Tables 1-2 to run (14..98)")
    ap.add_argument("--collisions", default="srt,mrt", help="paper form: srt, mrt or both")
    ap.add_argument("--eps", default="0.1",
                    help="paper form: initial perturbations delta/R0 to run (Fig. 2b uses 0.1, Fig. 3 "
                         "1/30, 0.05, 0.1)")
    ap.add_argument("--rho-ref", type=float, default=1.0,
                    help="reference density of the 16-bit deviation formats")
    ap.add_argument("--breakup-R0", type=float, default=32.0,
                    help="precision form: ligament radius of the run-to-break-up comparison")
    return ap.parse_args()


def workload(args):
    from paper_1905_09554_gb300 import inputs
    nx, ny, nz = inputs.ligament_box(args.R0, args.kR0)
    forcing = "shift" if args.collision == "srt" else "guo"
    rl, rv = inputs.COEXISTENCE[(forcing, -5.5, 1.0)]
    rule = f" ({args.mrt_rule} rule)" if args.collision == "mrt" else ""
    gtxt = "G=-5.5" if args.G2 == 0 else f"G1={-5.5 - args.G2:g} G2={args.G2:g} (two-belt force)"
    name = (f"ligament R0={args.R0:g} kR0={args.kR0:g} box {nx}x{ny}x{nz}, {gtxt}, "
            f"{args.collision.upper()}{rule} tau={args.tau:g}, {args.storage.upper()} populations, "
            f"5% cosine perturbation")
    return dict(nx=nx, ny=ny, nz=nz, rho_l=rl, rho_v=rv, name=name)


def mrt_rates(args):
    """Rates in moment order (rho e eps jx qx jy qy jz qz 3pxx 3pixx pww piww
    pxy pyz pxz mx my mz): the five shear moments at 1/tau, plus the energy
    moment for the paper's rule; the rest at 1.  None for SRT."""
    if args.collision != "mrt":
        return None
    s = [1.0] * 19
    for k in (9, 11, 13, 14, 15):
        s[k] = 1.0 / args.tau
    if args.mrt_rule == "paper":
        s[1] = 1.0 / args.tau
    return s


def host_info():
    """Host CPU of the run (model, architecture, logical CPUs)."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu": model or platform.processor() or None, "arch": platform.machine(),
            "logical_cpus": os.cpu_count()}


def measured_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock/throttle sampling every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if bus_id:
            cmd[1:1] = ["-i", bus_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.seek(0)
        text = self.out.read()
        os.unlink(self.out.name)
        return self.parse(text)

    @staticmethod
    def parse(text):
        """Median SM clock, maximum clock and the throttle reasons seen active
        in nvidia-smi's csv,noheader,nounits lines of FIELDS."""
        rows = [r.split(", ") for r in text.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# -------------------------------------------------------------- CPU oracle
def oracle_mlups(w, args, slab, min_seconds, max_steps):
    """FP64 reference step timed on the host cores on a z-slab (thickness
    `slab`, periodic) of the workload's initial state.  Returns
    (MLUPS, effective cores, description, steps)."""
    import numpy as np

    from oracle import lbm_oracle as o
    from paper_1905_09554_gb300 import inputs
    rho = inputs.ligament_density(w["nx"], w["ny"], slab, args.R0, 0.05, w["rho_l"], w["rho_v"])
    p = o.Params(G=-5.5, tau=args.tau, collision=args.collision, s=mrt_rates(args))
    f = o.init_populations(rho)
    f = o.step(f, p)  # warm-up
    t0, c0 = time.perf_counter(), os.times()
    steps = 0
    while steps < max_steps and (steps == 0 or time.perf_counter() - t0 < min_seconds):
        f = o.step(f, p)
        steps += 1
    dt = time.perf_counter() - t0
    c1 = os.times()
    cpu = (c1.user - c0.user) + (c1.system - c0.system)
    cells = rho.size
    assert np.isfinite(f).all()
    desc = (f"FP64 numpy oracle, {steps} steps of a {w['nx']}x{w['ny']}x{slab} periodic z-slab of the "
            f"workload's initial ligament ({cells} cells)")
    return cells * steps / dt / 1e6, max(1, round(cpu / dt)), desc, steps


def c_reference_mlups(w, args, slab, steps):
    """The OpenMP C reference (oracle/c/lbm_ref.c, SRT or MRT) on the same
    slab, all host threads: (MLUPS, threads, description), or None where it
    is not available (no C compiler, G2 != 0)."""
    if getattr(args, "G2", 0.0) != 0.0:
        return None
    try:
        from oracle import c_ref, lbm_oracle as o
        from paper_1905_09554_gb300 import inputs
        rho = inputs.ligament_density(w["nx"], w["ny"], slab, args.R0, 0.05, w["rho_l"], w["rho_v"])
        f = o.init_populations(rho)
        rates = mrt_rates(args)
        if rates is None:
            def run(k):
                return c_ref.run_srt(f, k, -5.5, args.tau)
        else:
            def run(k):
                return c_ref.run_mrt(f, k, -5.5, rates)
        run(1)  # build, load, warm up
        t0 = time.perf_counter()
        run(steps)
        dt = time.perf_counter() - t0
        n = c_ref.threads()
    except Exception:  # noqa: BLE001 - optional: no compiler or OpenMP on this host
        return None
    desc = (f"FP64 C reference with OpenMP ({n} threads), {steps} {args.collision.upper()} steps of the same "
            f"{w['nx']}x{w['ny']}x{slab} slab")
    return rho.size * steps / dt / 1e6, n, desc


# ------------------------------------------------------------ other forms
def measure_rate(storage, steps, warmup, R0=64.0, kR0=0.7, collision="srt", tau=1.0):
    """Device time per step (CUDA events on the lattice's stream around
    `steps` step launches) of the ligament R0, kR0 with `storage`
    populations; returns GLUPS, ms per step, cells and the launch shape."""
    import torch

    from paper_1905_09554_gb300 import inputs, lbm
    nx, ny, nz = inputs.ligament_box(R0, kR0)
    forcing = "shift" if collision == "srt" else "guo"
    rl, rv = inputs.COEXISTENCE[(forcing, -5.5, 1.0)]
    rates = None
    if collision == "mrt":
        rates = [1.0] * 19
        for k in (9, 11, 13, 14, 15):
            rates[k] = 1.0 / tau
    with lbm.Lattice(nx, ny, nz, G=-5.5, tau=tau, collision=collision, rates=rates, storage=storage) as L:
        L.init_ligament(R0, 0.05, rl, rv)
        L.step(warmup)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        L.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        cfg = L.kernel_config()
    cells = nx * ny * nz
    return {"glups": cells / (ms / 1e3) / 1e9, "ms_per_step": ms, "cells": cells, "kernel": cfg}


def breakup_run_to_pinch(storage, R0=16.0, kR0=0.7, collision="srt", tau=1.0, every=5, max_steps=20000):
    """Run the ligament R0, kR0 (5% perturbation, G = -5.5) to its first
    pinch-off, sampling the diagnostics every `every` steps; returns the
    break-up time in steps (interpolated; None if none within max_steps)
    and the density after 200 steps."""
    from paper_1905_09554_gb300 import diagnostics as dg
    from paper_1905_09554_gb300 import inputs, lbm
    nx, ny, nz = inputs.ligament_box(R0, kR0)
    forcing = "shift" if collision == "srt" else "guo"
    rl, rv = inputs.COEXISTENCE[(forcing, -5.5, 1.0)]
    with lbm.Lattice(nx, ny, nz, G=-5.5, tau=tau, collision=collision, storage=storage) as L:
        L.init_ligament(R0, 0.05, rl, rv)
        L.step(200)
        rho200 = L.density()
        ts, mins, t = [], [], 200
        while t <= max_steps:
            d = L.diag(rl, rv, raise_nonfinite=False)
            ts.append(t)
            mins.append(float(d["maxrho_z"].min()))
            if mins[-1] < 0.5 * (rl + rv) or d["status"] != 0:
                break
            L.step(every)
            t += every
    return dg.breakup_time(ts, mins, rl, rv), rho200


def measure_forms(device, clocks):
    """The forms named beside the headline metric, each against the plain
    FP64 single-ligament step: FP64, FP16 / FP16-local rates on the headline
    box; FP32 / FP16-local / BF16-local accuracy over a break-up run
    (R0 = 16); the batched form; the adjoint form.  About half a minute."""
    peak = measured_hbm()[0]
    forms = {"rates_workload": "ligament R0=64 kR0=0.7 box 256x256x575, G=-5.5, SRT tau=1 (device time, CUDA "
                               "events around the step launches)",
             "accuracy_workload": "ligament R0=16 kR0=0.7 box 64x64x144, G=-5.5, SRT tau=1, 5% perturbation, "
                                  "run to the first pinch-off, diagnostics every 5 steps; errors against the "
                                  "FP64 GPU run of the same case"}
    f64 = measure_rate("f64", steps=20, warmup=3)
    rec = step_record()
    fpc = rec.get("fp64_flops_per_cell") if rec else None
    pk, src = fp64_peak(device, clocks)
    forms["f64"] = {"glups": f64["glups"], "ms_per_step": f64["ms_per_step"],
                    "hbm_frac": 304 * f64["glups"] / peak,
                    "fp64_pipe_frac": (fpc * f64["glups"] / 1e3 / pk) if fpc else None,
                    "fp64_flops_per_cell": fpc, "fp64_peak_tflops": pk, "fp64_peak_source": src,
                    "kernel": f64["kernel"]}
    for st, bpc in (("f16l", 84), ("f16", 76), ("bf16l", 84)):
        r = measure_rate(st, steps=100, warmup=5)
        forms[st] = {"glups": r["glups"], "ms_per_step": r["ms_per_step"], "bytes_per_cell": bpc,
                     "hbm_frac": bpc * r["glups"] / peak, "speedup_vs_f64": r["glups"] / f64["glups"],
                     "kernel": r["kernel"]}
    import numpy as np
    tb64, rho64 = breakup_run_to_pinch("f64")
    forms["f64"]["t_break_steps_R0_16"] = tb64
    for st in ("f32", "f16l", "bf16l"):
        tb, rho = breakup_run_to_pinch(st)
        forms.setdefault(st, {})
        forms[st]["t_break_steps_R0_16"] = tb
        forms[st]["t_break_rel_err_vs_f64"] = abs(tb - tb64) / tb64 if tb and tb64 else None
        forms[st]["max_abs_rho_err_200_vs_f64"] = float(np.abs(rho - rho64).max())
    b = measure_batched(300, 10)
    forms["batched"] = {"ligaments_per_s": b["ligaments_per_s"], "aggregate_glups": b["aggregate_mlups"] / 1e3,
                        "hbm_frac": b["hbm_gbs"] / peak, "speedup_vs_f64": b["aggregate_mlups"] / 1e3 / f64["glups"],
                        "cells": b["cells"], "tile_y": b["config"]["tile_y"], "zchunk": b["config"]["zchunk"],
                        "workload": "64 ligaments R0 in {8,12,16}, kR0 ~ U[0.2,1.0) seed 0, FP32 SRT; ligaments/s "
                                    "of 3000-step runs from 300 timed steps"}
    adj = measure_adjoint()
    a, d = adj["f32"], adj["f64"]
    forms["adjoint"] = {"f32_adjoint_steps_per_s": adj["T"] / a["bwd_s"],
                        "f64_adjoint_steps_per_s": adj["T"] / d["bwd_s"],
                        "f32_forward_with_checkpoints_steps_per_s": adj["T"] / a["fwd_s"],
                        "f32_vs_f64_gradient": adj["fp32_vs_fp64"],
                        "step_launch_shape": {"f32": adj["f32_tune"], "f64": adj["f64_tune"]},
                        "workload": "64x64x180 ligament, neck energy at step 500, checkpoints every 23"}
    return forms


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args)
    # each step on a 1-cell-thick slab (65536 cells) keeps K+W steps within minutes
    cells_xy = w["nx"] * w["ny"]
    per_step = cells_xy * 1.5e-6
    slab = max(1, min(16, int(150.0 / max(1, args.steps + args.warmup) / per_step)))
    from oracle import lbm_oracle as o
    from paper_1905_09554_gb300 import inputs
    rho = inputs.ligament_density(w["nx"], w["ny"], slab, args.R0, 0.05, w["rho_l"], w["rho_v"])
    p = o.Params(G=-5.5, tau=args.tau, collision=args.collision, s=mrt_rates(args))
    f = o.init_populations(rho)
    for _ in range(args.warmup):
        f = o.step(f, p)
    t0, c0 = time.perf_counter(), os.times()
    for _ in range(args.steps):
        f = o.step(f, p)
    dt = time.perf_counter() - t0
    c1 = os.times()
    cores = max(1, round(((c1.user - c0.user) + (c1.system - c0.system)) / dt))
    value = rho.size * args.steps / dt / 1e6
    sample = (f"FP64 numpy oracle; each step is a {w['nx']}x{w['ny']}x{slab} periodic z-slab "
              f"({rho.size} cells) of the workload's initial ligament")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w["name"], "sample_cells": rho.size},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "host": host_info(),
    }), flush=True)


# --------------------------------------------------------------- multi-rank
def max_over_ranks(x, dist=None):
    """Maximum of a per-rank float over all ranks (NCCL: on the rank's GPU;
    gloo: on the host).  With no process group, x itself."""
    if dist is None or not dist.is_initialized():
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(cells_per_rank, steps, max_ms, world):
    """MLUPS of the whole job: every rank advances its own replica of
    cells_per_rank cells by `steps` steps; the job takes the slowest rank's
    time."""
    return world * cells_per_rank * steps / (max_ms / 1e3) / 1e6


# ------------------------------------------------------------------- GPU arm
def run_ours(args):
    import numpy as np
    import torch

    from paper_1905_09554_gb300 import lbm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    w = workload(args)
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    ncell = nx * ny * nz
    L = lbm.Lattice(nx, ny, nz, G=-5.5 - args.G2, G2=args.G2, tau=args.tau, collision=args.collision,
                    storage=args.storage,
                    rates=mrt_rates(args), zchunk=args.zchunk, tile_y=args.tile_y, kernel=args.kernel)
    L.init_ligament(args.R0, 0.05, w["rho_l"], w["rho_v"])
    L_info = L.kernel_config()
    stream = torch.cuda.current_stream()
    d0 = L.diag(w["rho_l"], w["rho_v"])
    L.step(args.warmup)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    bus = None
    try:
        bus = torch.cuda.get_device_properties(local).pci_bus_id
    except Exception:
        bus = None
    sampler = ClockSampler(bus) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    t_start.record(stream)
    for s, e in ev:
        s.record(stream)
        L.step(1)
        e.record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    total_ms = t_start.elapsed_time(t_end)
    kernel_ms = sum(s.elapsed_time(e) for s, e in ev) / args.steps
    d1 = L.diag(w["rho_l"], w["rho_v"])
    mass_drift = abs(d1["mass"] - d0["mass"]) / d0["mass"]

    total_ms = max_over_ranks(total_ms, dist)
    value = whole_job_mlups(ncell, args.steps, total_ms, world)

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        K = args.e2e_steps
        rho_host = torch.empty((nz, ny, nx), dtype=torch.float64, pin_memory=True)
        from paper_1905_09554_gb300 import inputs
        rho_host.numpy()[...] = inputs.ligament_density(nx, ny, nz, args.R0, 0.05, w["rho_l"], w["rho_v"])
        rho_out = torch.empty((nz, ny, nx), dtype=torch.float64, pin_memory=True)
        diag_every = args.e2e_diag_every
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        L.set_density(rho_host.numpy())
        for k in range(0, K, diag_every):
            L.step(min(diag_every, K - k))
            L.diag(w["rho_l"], w["rho_v"])
        lbm.lbm_moments(L.ctx, rho_out.data_ptr(), None, None, None, 0)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, dist)
        n_diag = (K + diag_every - 1) // diag_every
        e2e = {"value": world * ncell * K / dt / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 8 * ncell / K,
               "d2h_bytes_per_step": (8 * ncell + n_diag * 8 * (4 + 2 * nz)) / K,
               "steps": K, "diag_every": diag_every}
    L.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peak, src = measured_hbm()
    bpc = 2 * 19 * BYTES_PER_POP[args.storage] + EXTRA_BYTES_PER_CELL.get(args.storage, 0)
    kname = KERNEL_NAMES.get(L_info["kernel"], "sc_step_kernel")
    rec = step_record()
    if args.storage == "f64" and rec and rec.get("fp64_flops_per_cell"):
        # FP64 is bound by the FP64 pipe: SMs x 2 FP64 lanes per clock
        # (ncu's peak_sustained) x SM clock x 2 flops per FMA.
        fpc = rec["fp64_flops_per_cell"]
        achieved = fpc * ncell / (kernel_ms / 1e3) / 1e12
        peak_alu, peak_src = fp64_peak(local, clocks)
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak_alu, "unit": "TFLOP/s",
                    "frac": achieved / peak_alu, "traffic": load_traffic(args, ncell, L_info, (nx, ny, nz)),
                    "peak_source": peak_src,
                    "kernel": kname, "fp64_flops_per_cell": fpc, "kernel_ms": kernel_ms,
                    "hbm_frac": bpc * ncell / (kernel_ms / 1e3) / 1e9 / peak}
    else:
        achieved = bpc * ncell / (kernel_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": load_traffic(args, ncell, L_info, (nx, ny, nz)),
                    "peak_source": f"{src} HBM copy bandwidth",
                    "kernel": kname, "algorithmic_bytes_per_cell": bpc, "kernel_ms": kernel_ms}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        mlups, cores, desc, _ = oracle_mlups(w, args, slab=16, min_seconds=10.0, max_steps=20)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": desc}
        c_res = c_reference_mlups(w, args, slab=16, steps=40)
        if c_res is not None:  # the same method in plain C on every host thread
            cpu["openmp_c_reference"] = {"value": c_res[0], "unit": "MLUPS", "threads": c_res[1],
                                         "sample": c_res[2]}

    forms = None
    if not args.no_forms and world == 1:
        forms = measure_forms(local, clocks)

    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": {"workload": w["name"], "cells": ncell, "collision": args.collision,
                   "storage": args.storage, "parallelism": f"replicas x{world}",
                   "kernel": L_info["kernel"], "zchunk": L_info["zchunk"], "tile_y": L_info["tile_y"],
                   "grid": L_info["grid"],
                   "l2": "inputs larger than L2 (two population copies of "
                         f"{19 * BYTES_PER_POP[args.storage] * ncell / 1e9:.2f} GB each)",
                   "mass_rel_drift": mass_drift},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": args.steps, "host": host_info(), "forms": forms,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def fp64_peak(device, clocks=None):
    """FP64 pipe peak in TFLOP/s: the device's SM count x 2 FP64 lanes per SM
    and clock (ncu's peak_sustained for the FP64 pipe on GB300) x the median
    SM clock sampled under load (else the maximum clock) x 2 flops per FMA."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz")
    src = "sampled median SM clock"
    if not mhz:
        try:
            mhz = float(subprocess.run(["nvidia-smi", "-i", str(device), "--query-gpu=clocks.max.sm",
                                        "--format=csv,noheader,nounits"], capture_output=True,
                                       text=True, timeout=10).stdout.split()[0])
            src = "maximum SM clock"
        except Exception:  # noqa: BLE001
            mhz, src = 2070.0, "nominal maximum SM clock"
    peak = sms * 2 * mhz * 1e6 * 2 / 1e12
    return peak, f"FP64 pipe: {sms} SMs x 2 lanes/clk x {mhz:.0f} MHz ({src}) x 2 flop (derived)"


STEP_SOURCES = ("step_kernel.cuh", "codec.cuh", "lattice.cuh", "step_multirange.cuh", "e8.cuh", "step_pair16.cuh")


def step_record():
    """The committed ncu record for the current step-kernel source, or None
    once the kernel has changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "step_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh)
    h = hashlib.sha256()
    for f in STEP_SOURCES:
        with open(os.path.join(ROOT, "paper_1905_09554_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return rec if rec.get("kernel_sha256") == h.hexdigest() else None


def traffic_key(dims, args, info):
    nx, ny, nz = dims
    return (f"{nx}x{ny}x{nz}_{args.collision}_{args.storage}_tau{args.tau:g}_k{info['kernel']}"
            f"_ty{info['tile_y']}_zc{info['zchunk']}")


def load_traffic(args, ncell, info, dims=None):
    """DRAM bytes per launch from the committed ncu record, if it was taken on
    the current kernel source, this box and this collision/storage/tau/launch
    shape (kernel variant, tile height, z-chunk length)."""
    rec = step_record()
    if rec is None or dims is None:
        return None
    key = traffic_key(dims, args, info)
    per = rec.get("bytes_per_cell", {}).get(key)
    return per * ncell if per is not None else None


def measure_batched(steps, warmup, trial_steps=3):
    """64 independent ligaments (R0 in {8, 12, 16}, kR0 uniform on [0.2, 1.0)
    from seed 0, box 4R0 x 4R0 x round(2 pi R0 / kR0)), FP32 SRT tau = 1,
    G = -5.5, 3% perturbation, advanced together by one launch per step
    (pairs of steps from a CUDA graph) after the launch-shape autotuner.
    Returns the device time of `steps` steps and the chosen configuration."""
    import torch

    from paper_1905_09554_gb300 import inputs, lbm
    insts = inputs.batch_instances(64, seed=0)
    dims = [(d["nx"], d["ny"], d["nz"]) for d in insts]
    rl, rv = inputs.COEXISTENCE[("shift", -5.5, 1.0)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        B = lbm.Batch(dims, G=-5.5, tau=1.0, collision="srt", storage="f32", stream=stream.cuda_stream)
        best = B.tune(trial_steps=trial_steps)
        for box, d in zip(B.boxes, insts):
            box.init_ligament(d["R0"], 0.03, rl, rv)
        B.step(warmup)
        cfg = B.config()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        B.step(steps)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        B.close()
    cells = cfg["cells"]
    return {"ms": ms, "steps": steps, "cells": cells, "config": cfg, "tune": best,
            "ligaments_per_s": 64.0 / (ms / 1e3 * 3000.0 / steps),
            "aggregate_mlups": cells * steps / (ms / 1e3) / 1e6,
            "hbm_gbs": 152 * cells / (ms / steps / 1e3) / 1e9}


def run_batched(args):
    """The batched form: `value` is ligaments/s, complete runs of 3000 steps
    per second, measured over --steps steps."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    m = measure_batched(args.steps, args.warmup)
    cfg = m["config"]
    peak = measured_hbm()[0]
    line = {
        "metric": "batched ligaments/s (64 uneven ligaments, one launch per step)",
        "value": m["ligaments_per_s"],
        "unit": "ligaments/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": m["ms"] / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "64 ligaments, R0 in {8,12,16}, kR0 ~ U[0.2,1.0) seed 0, boxes 4R0x4R0xround(2piR0/kR0), "
                               "G=-5.5, SRT tau=1, FP32, 3% perturbation",
                   "cells": m["cells"], "tile_y": cfg["tile_y"], "zchunk": cfg["zchunk"], "grid": cfg["grid"],
                   "autotune_ms_per_step": m["tune"]["ms_per_step"]},
        "aggregate_mlups": m["aggregate_mlups"],
        "roofline": {"bound": "hbm", "achieved": m["hbm_gbs"], "peak": peak, "unit": "GB/s",
                     "frac": m["hbm_gbs"] / peak},
        "gpu_launches": args.steps,
    }
    print(json.dumps(line), flush=True)


def golden_sigma(forcing):
    path = os.path.join(ROOT, "tests", "golden", "sigma.json")
    try:
        with open(path) as fh:
            return [c for c in json.load(fh)["cases"] if c["forcing"] == forcing][0]["sigma"]
    except Exception:
        return None


def measure_adjoint(T=500, every=23):
    """Gradient of the neck energy J = mean_z (R(z) - mean R)^2 at step T with
    respect to the initial density, G and tau, for the 64 x 64 x 180
    ligament (R0 = 16, kR0 = 0.56, 5% perturbation plus N(0, 1e-3) per-cell
    noise from seed 1), SRT tau = 1, G = -5.5, checkpoints every `every`
    steps, with FP32 and with FP64 populations.  Returns per precision the
    objective, the gradients and the forward / backward wall times."""
    import numpy as np
    import torch

    from paper_1905_09554_gb300 import inputs, lbm
    nx, ny, nz = 64, 64, 180
    R0 = 16.0
    rl, rv = inputs.COEXISTENCE[("shift", -5.5, 1.0)]
    rho0 = inputs.noisy_ligament_density(nx, ny, nz, R0, 0.05, rl, rv, 1e-3, seed=1)

    def dJ(rho):
        A = ((rho - rv) / (rl - rv)).sum(axis=(1, 2))
        R = np.sqrt(A / np.pi)
        g = (2.0 / nz) * (R - R.mean()) / (2.0 * np.pi * R * (rl - rv))
        return np.broadcast_to(g[:, None, None], rho.shape).copy(), float(((R - R.mean()) ** 2).mean())

    out = {}
    for storage in ("f32", "f64"):
        with lbm.Lattice(nx, ny, nz, G=-5.5, tau=1.0, storage=storage) as L:
            # the recomputation steps this small box many times: pick its launch shape
            out[storage + "_tune"] = L.tune(trial_steps=4)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            L.adjoint_forward(rho0, T, every)
            r, _ = L.moments()
            t1 = time.perf_counter()
            g, J = dJ(r)
            t2 = time.perf_counter()
            grad, gG, gT = L.adjoint_backward(g)
            t3 = time.perf_counter()
        out[storage] = dict(J=J, grad=grad, dG=gG, dtau=gT, fwd_s=t1 - t0, bwd_s=t3 - t2)
    a, b = out["f32"], out["f64"]
    out["fp32_vs_fp64"] = {"dJ_dG_rel": abs(a["dG"] - b["dG"]) / abs(b["dG"]),
                           "dJ_dtau_rel": abs(a["dtau"] - b["dtau"]) / abs(b["dtau"]),
                           "dJ_drho0_maxabs_rel": float(np.abs(a["grad"] - b["grad"]).max()
                                                        / np.abs(b["grad"]).max())}
    out["cells"], out["T"], out["every"] = nx * ny * nz, T, every
    return out


def run_adjoint(args):
    """The adjoint form (see measure_adjoint): `value` is adjoint steps/s of
    the FP32 backward pass (which includes recomputing each segment from its
    checkpoint); the FP64 gradient of the same problem is the accuracy
    reference."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    out = measure_adjoint()
    a, b, T = out["f32"], out["f64"], out["T"]
    line = {
        "metric": "adjoint steps/s (SRT, 64x64x180, 500 steps, checkpoints every 23)",
        "value": T / a["bwd_s"], "unit": "adjoint steps/s", "n_gpus": 1, "steps": T, "warmup": 0,
        "ms_per_step": a["bwd_s"] / T * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "ligament 64x64x180, R0=16, kR0=0.56, 5% perturbation + N(0,1e-3) noise seed 1, "
                               "G=-5.5, SRT tau=1, objective: neck energy at step 500",
                   "checkpoint_every": out["every"], "cells": out["cells"]},
        "forward_with_checkpoints_steps_per_s": T / a["fwd_s"],
        "step_launch_shape": {"f32": out["f32_tune"], "f64": out["f64_tune"]},
        "fp64": {"adjoint_steps_per_s": T / b["bwd_s"], "dJ_dG": b["dG"], "dJ_dtau": b["dtau"], "J": b["J"]},
        "fp32": {"dJ_dG": a["dG"], "dJ_dtau": a["dtau"], "J": a["J"]},
        "fp32_vs_fp64": out["fp32_vs_fp64"],
    }
    print(json.dumps(line), flush=True)


def run_precision(args):
    """Population storage formats against the FP64 run (MRT, G = -5.5,
    tau = 1, shear rule): max-abs rho and u error after 200 steps of the
    R0 = --R0 ligament (kR0 = 0.7, 5% perturbation), and the growth rate and
    break-up time of the R0 = --breakup-R0 ligament run to break-up."""
    import numpy as np
    import torch

    from paper_1905_09554_gb300 import diagnostics as dg
    from paper_1905_09554_gb300 import inputs, lbm
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rl, rv = inputs.COEXISTENCE[("guo", -5.5, 1.0)]
    rates = [1.0] * 19  # shear rule at tau = 1: every rate is 1
    sig = golden_sigma("guo")
    fmts = ["f64", "f32", "f16", "bf16", "f16l", "bf16l"]
    res = {f: {} for f in fmts}
    nx, ny, nz = inputs.ligament_box(args.R0, args.kR0)
    fields = {}
    for f in fmts:
        with lbm.Lattice(nx, ny, nz, G=-5.5, tau=1.0, collision="mrt", rates=rates, storage=f,
                         rho_ref=args.rho_ref) as L:
            L.init_ligament(args.R0, 0.05, rl, rv)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            stream = torch.cuda.current_stream()
            torch.cuda.synchronize()
            e0.record(stream)
            L.step(200)
            e1.record(stream)
            torch.cuda.synchronize()
            res[f]["mlups_200"] = nx * ny * nz * 200 / (e0.elapsed_time(e1) / 1e3) / 1e6
            res[f]["kernel"] = L.kernel_config()
            fields[f] = L.moments()
    for f in fmts[1:]:
        res[f]["err200_rho"] = float(np.abs(fields[f][0] - fields["f64"][0]).max())
        res[f]["err200_u"] = float(np.abs(fields[f][1] - fields["f64"][1]).max())
    del fields
    R0b = args.breakup_R0
    bx, by, bz = inputs.ligament_box(R0b, args.kR0)
    tcap = math.sqrt(rl * R0b ** 3 / sig) if sig else 1000.0
    every = 20
    for f in fmts:
        with lbm.Lattice(bx, by, bz, G=-5.5, tau=1.0, collision="mrt", rates=rates, storage=f,
                         rho_ref=args.rho_ref) as L:
            L.init_ligament(R0b, 0.05, rl, rv)
            ts, amps, mins = [], [], []
            t = 0
            while t <= 60 * tcap:
                d = L.diag(rl, rv, raise_nonfinite=False)
                ts.append(t)
                amps.append(dg.mode_amplitude(d["area_z"]))
                mins.append(float(d["maxrho_z"].min()))
                if mins[-1] < 0.5 * (rl + rv) or d["status"] != 0:
                    break
                L.step(every)
                t += every
        tb = dg.breakup_time(ts, mins, rl, rv)
        w = dg.growth_rate(ts, amps, t_start=tcap, a_stop=0.3 * R0b)
        res[f]["t_break"] = tb
        res[f]["t_break_over_tcap"] = tb / tcap if tb is not None else None
        res[f]["growth_rate_x_tcap"] = w * tcap if w is not None else None
    for f in fmts[1:]:
        ref = res["f64"]
        res[f]["t_break_rel_err"] = (abs(res[f]["t_break"] - ref["t_break"]) / ref["t_break"]
                                     if res[f]["t_break"] and ref["t_break"] else None)
        res[f]["growth_rel_err"] = (abs(res[f]["growth_rate_x_tcap"] - ref["growth_rate_x_tcap"])
                                    / ref["growth_rate_x_tcap"]
                                    if res[f]["growth_rate_x_tcap"] and ref["growth_rate_x_tcap"] else None)
    line = {
        "metric": "storage precision vs FP64 (MRT Guo, G=-5.5, tau=1)",
        "value": res["f32"]["err200_rho"], "unit": "max|rho - rho_FP64| after 200 steps (FP32)",
        "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
        "config": {"workload_200": f"ligament R0={args.R0:g} kR0={args.kR0:g} box {nx}x{ny}x{nz}",
                   "workload_breakup": f"ligament R0={R0b:g} kR0={args.kR0:g} box {bx}x{by}x{bz}, "
                                       f"diagnostics every {every} steps, t_cap={tcap:.1f}",
                   "rho_ref": args.rho_ref, "dev_scale": 1.0},
        "formats": res,
    }
    print(json.dumps(line), flush=True)


def run_paper(args):
    """The paper's break-up experiment (Sec. 3-4, Tables 1-2, Fig. 2b) at its
    own parameters: G0 = -5.3, Oh = 0.1, tau / rho_l / rho_v / t_cap of Table 1
    (SRT) or Table 2 (MRT, rates of Sec. 2), a box Ly x Ly x Lx with two
    wavelengths of a perturbation eps = delta/R0 along the ligament (the
    paper's x axis is this code's z axis), FP32 populations, tanh profile of
    width 2.  Runs until the ligament breaks (min over slices of max rho below
    the mid density) and reports T_break / t_cap beside the paper's value
    (Fig. 2b at eps = 0.1; Fig. 3's points at R0 = 98) and Fig. 3's linear
    stability curve."""
    import numpy as np
    import torch

    from paper_1905_09554_gb300 import experiments as ex
    from paper_1905_09554_gb300 import lbm
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    gold = os.path.join(ROOT, "tests", "golden")
    tables = {"srt": np.loadtxt(os.path.join(gold, "paper_table1_srt.txt")),
              "mrt": np.loadtxt(os.path.join(gold, "paper_table2_mrt.txt"))}
    fig = np.loadtxt(os.path.join(gold, "paper_fig2b_breakup.txt"))
    fig3 = np.loadtxt(os.path.join(gold, "paper_fig3_points.txt"))
    lsa = np.loadtxt(os.path.join(gold, "paper_fig3_lsa.txt"))
    radii = [int(r) for r in args.radii.split(",") if r]
    epss = [float(e) for e in args.eps.split(",") if e]
    cases = []
    for coll, R0, eps in [(c, r, e) for c in args.collisions.split(",") if c for r in radii for e in epss]:
        ic = 0 if coll == "srt" else 1
        row = [r for r in tables[coll] if int(r[0]) == R0][0]
        _, Lx, Ly, tau, tcap, rl, rv, sigma = row
        nx, ny, nz = int(Ly), int(Ly), int(Lx)
        # the paper's value for this case: Fig. 2b at eps = 0.1, Fig. 3's points at R0 = 98
        fig_t, fig_sat = None, None
        if abs(eps - 0.1) < 1e-9:
            fig_t, fig_sat = [(f[2], int(f[3])) for f in fig if int(f[0]) == ic and int(f[1]) == R0][0]
        elif R0 == 98:
            hit = [f[2] for f in fig3 if int(f[0]) == ic and abs(f[1] - eps) < 1e-6]
            fig_t = hit[0] if hit else None
        # linear stability analysis of the figure (kR0 = 0.687 and Oh = 0.1 at every radius)
        lsa_t = float(np.interp(eps, lsa[:, 0], lsa[:, 1])) if lsa[0, 0] <= eps <= lsa[-1, 0] else None
        every = max(1, int(tcap / 40))
        with lbm.Lattice(nx, ny, nz, G=-5.3, tau=tau, collision=coll, storage="f32") as L:
            L.init_ligament(float(R0), eps, rl, rv, n_waves=2)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ck = None
            if args.checkpoint_dir:
                os.makedirs(args.checkpoint_dir, exist_ok=True)
                ck = os.path.join(args.checkpoint_dir, f"paper_{coll}_R{R0:g}_eps{eps:g}.ckpt")
            res = ex.breakup_run(L, R0, tcap, rl, rv, every, series=args.series, components=args.components,
                                 checkpoint=ck)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            cfg = L.kernel_config()
        tb = res["T_break_over_tcap"]
        cases.append({"collision": coll, "R0": R0, "eps": eps, "box": [nx, ny, nz], "tau": tau, "t_cap": tcap,
                      "rho_l": rl, "rho_v": rv, "steps": res["steps"], "diag_every": every,
                      "drops_max": res["drops_max"], "drops_final": res["drops_final"],
                      "satellites": res["satellites"], "satellites_transient": res["satellites_transient"],
                      "drops_3d": res.get("drops_3d"), "satellites_3d": res.get("satellites_3d"),
                      "paper_satellites": fig_sat, "T_break_over_tcap": tb,
                      "paper_T_break": fig_t, "lsa_T_break": lsa_t,
                      "rel_diff": (tb - fig_t) / fig_t if tb is not None and fig_t else None,
                      "resumed_from_step": res["resumed_from_step"], "wall_s": wall,
                      "glups": nx * ny * nz * (res["steps"] - res["resumed_from_step"]) / wall / 1e9,
                      "kernel": cfg})
        if "series" in res:
            cases[-1]["series"] = res["series"]
            print(json.dumps({"collision": coll, "R0": R0, "eps": eps,
                              "pinch_linear_fit": res["series"]["pinch_linear_fit"],
                              "velocity_at_t_star": res["series"]["velocity_at_t_star"]}), flush=True)
        print(json.dumps(cases[-1]), flush=True)
    print(json.dumps({"metric": "paper break-up experiment (Fig. 2b) at the paper's parameters",
                      "unit": "T_break / t_cap", "data": "synthetic", "cases": cases}), flush=True)


def run_calibrate(args):
    """The calibration of Sec. 3 at G0 = -5.3, Oh = 0.1, measured with the GPU
    step: SRT iterates tau -> (Laplace test on droplets of radius 16, 20, 24
    in boxes of 4 R, flat slab) -> the tau that meets Oh, from --tau0 until
    two consecutive sigma agree to --cal-tol; MRT (rates of Sec. 2) takes one
    pass at Table 2's tau.  Reports tau, sigma, rho_l, rho_v and t_cap beside
    Tables 1 and 2."""
    import numpy as np
    import torch

    from paper_1905_09554_gb300 import calibration as cal
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    gold = os.path.join(ROOT, "tests", "golden")
    tables = {"srt": np.loadtxt(os.path.join(gold, "paper_table1_srt.txt")),
              "mrt": np.loadtxt(os.path.join(gold, "paper_table2_mrt.txt"))}
    radii = [int(r) for r in args.radii.split(",") if r]
    G = -5.3
    cases = []
    cache = {}

    def measure(coll, tau):
        key = (coll, round(tau, 6))
        if key not in cache:
            rl, rv, _ = cal.flat_coexistence(G, tau, coll, storage="f64")
            lap = cal.laplace_sigma(G, tau, coll, rho_guess=(rl, rv))
            cache[key] = (lap["sigma"], rl, rv, lap["fit_r2"])
        return cache[key]

    t0 = time.perf_counter()
    for coll in [c for c in args.collisions.split(",") if c]:
        for R0 in radii:
            row = [r for r in tables[coll] if int(r[0]) == R0][0]
            _, Lx, Ly, tau_t, tcap_t, rl_t, rv_t, sig_t = row
            if coll == "srt":
                out = cal.calibrate_tau(R0, lambda t: measure("srt", t)[:2], tau0=args.tau0, rel_tol=args.cal_tol)
                tau = out["tau"]
                iters = out["iterations"]
            else:
                tau, iters = tau_t, 1
            sig, rl, rv, r2 = measure(coll, tau)
            tc = cal.t_cap(sig, rl, R0)
            cases.append({"collision": coll, "R0": R0, "tau": tau, "iterations": iters,
                          "tau_for_oh": cal.tau_for_oh(0.1, sig, rl, R0),
                          "sigma": sig, "rho_l": rl, "rho_v": rv, "t_cap": tc, "laplace_fit_r2": r2,
                          "table": {"tau": tau_t, "sigma": sig_t, "rho_l": rl_t, "rho_v": rv_t, "t_cap": tcap_t},
                          "rel_diff": {"tau_minus_half": (tau - 0.5) / (tau_t - 0.5) - 1, "sigma": sig / sig_t - 1,
                                       "rho_l": rl / rl_t - 1, "rho_v": rv / rv_t - 1, "t_cap": tc / tcap_t - 1}})
            print(json.dumps(cases[-1]), flush=True)
    print(json.dumps({"metric": "Sec. 3 calibration (Laplace test, flat interface, Oh = 0.1) vs Tables 1-2",
                      "unit": "relative difference", "data": "synthetic", "G": G,
                      "wall_s": time.perf_counter() - t0, "cases": cases}), flush=True)


def run_multirange(args):
    """The two-belt (multirange) force that Sec. 2 names: for splits of
    G1 + G2 = -5.5 (MRT, every rate 1), the flat-interface coexistence
    densities, the bulk-pressure balance with P = rho cs2 + cs2 (G1 + G2)
    psi^2 / 2, and the Laplace-test surface tension (droplets of radius 16,
    20, 24, FP32); then the step rate of the two-belt kernel on the
    256 x 256 x 575 ligament (G1 = -7, G2 = 1.5, SRT tau = 1, FP32)."""
    import torch

    from paper_1905_09554_gb300 import calibration as cal
    from paper_1905_09554_gb300 import lbm
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    splits = []
    for G1, G2 in ((-5.5, 0.0), (-7.0, 1.5), (-4.5, -1.0), (-3.5, -2.0)):
        rl, rv, st = cal.flat_coexistence(G1, 1.0, "mrt", G2=G2, rho_guess=(2.25, 0.06))
        lap = cal.laplace_sigma(G1, 1.0, "mrt", G2=G2, rho_guess=(rl, rv), storage="f32", tol=1e-6)
        pl, pv = float(cal.pressure(rl, G1, G2=G2)), float(cal.pressure(rv, G1, G2=G2))
        splits.append({"G1": G1, "G2": G2, "rho_l": rl, "rho_v": rv, "pressure_l": pl, "pressure_v": pv,
                       "sigma": lap["sigma"], "laplace_fit_r2": lap["fit_r2"]})
        print(json.dumps(splits[-1]), flush=True)
    base = splits[0]["sigma"]
    for s_ in splits:
        s_["sigma_rel_to_single_belt"] = s_["sigma"] / base - 1
    nx, ny, nz = 256, 256, 575
    L = lbm.Lattice(nx, ny, nz, G=-7.0, G2=1.5, tau=1.0, collision="srt", storage="f32")
    L.init_ligament(64, 0.05, 2.24, 0.05)
    L.step(args.warmup)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 200))
    torch.cuda.synchronize()
    e0.record(stream)
    L.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    cfg = L.kernel_config()
    L.close()
    print(json.dumps({
        "metric": "two-belt Shan-Chen force: surface tension at fixed EoS, and step rate",
        "value": nx * ny * nz / (ms / 1e3) / 1e6, "unit": "MLUPS", "n_gpus": 1, "steps": steps,
        "ms_per_step": ms, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "ligament R0=64 kR0=0.7 box 256x256x575, G1=-7, G2=1.5, SRT tau=1, FP32",
                   "kernel": cfg},
        "roofline": {"bound": "hbm", "achieved": 152 * nx * ny * nz / (ms / 1e3) / 1e9,
                     "peak": measured_hbm()[0], "unit": "GB/s"},
        "splits": splits}), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.form == "batched":
        run_batched(args)
    elif args.form == "adjoint":
        run_adjoint(args)
    elif args.form == "precision":
        run_precision(args)
    elif args.form == "paper":
        run_paper(args)
    elif args.form == "calibrate":
        run_calibrate(args)
    elif args.form == "multirange":
        run_multirange(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
