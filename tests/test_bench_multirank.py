"""bench.py's multi-rank host logic (replicas: max-over-ranks timing and the
whole-job MLUPS) with two gloo ranks on the CPU."""

import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 * (rank + 1)  # rank 1 is the slow one
    m = bench.max_over_ranks(ms, dist)
    out[rank] = (m, bench.whole_job_mlups(1_000_000, 100, m, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    port = 29500 + os.getpid() % 2000
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0
    # 2 replicas x 1e6 cells x 100 steps in 20 ms = 10000 MLUPS
    assert abs(res[0][1] - 10000.0) < 1e-9


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_mlups(37_683_200, 2000, 1000.0, 1) == pytest.approx(75366.4)


def test_clock_parser_reads_only_active_reasons():
    sys.path.insert(0, ROOT)
    import bench
    text = "\n".join([
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    ])
    got = bench.ClockSampler.parse(text)
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.ClockSampler.parse("") is None


def test_traffic_record_lookup_by_kernel_source_and_launch_shape():
    """The committed ncu record is used only for the kernel sources it was
    taken on and for a matching collision / storage / tau / launch shape."""
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    rec = bench.step_record()
    if rec is None:
        pytest.skip("profiles/step_traffic.json was taken on other kernel sources")
    args = argparse.Namespace(collision="srt", storage="f32", tau=1.0)
    info = {"kernel": 3, "tile_y": 16, "zchunk": 32}
    n = 37_683_200
    dims = (256, 256, 575)
    per_cell = rec["bytes_per_cell"]["256x256x575_srt_f32_tau1_k3_ty16_zc32"]
    assert 152.0 <= per_cell < 160.0
    assert bench.load_traffic(args, n, info, dims) == pytest.approx(per_cell * n)
    assert bench.load_traffic(args, n, dict(info, zchunk=58), dims) is None
    assert bench.load_traffic(args, n, info, (256, 256, 576)) is None


def test_reference_arm_prints_the_contract_line_and_other_ranks_stay_silent():
    """`bench.py --impl reference` times the oracle on the host and prints one
    JSON line with the contract's keys; a rank other than 0 prints nothing."""
    import json
    import subprocess

    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, RANK="0")
    out = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0 and d["higher_is_better"]
    assert "workload" in d["config"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert set(d["e2e"]) == {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert d["host"]["logical_cpus"] >= 1 and d["host"]["arch"]
    out1 = subprocess.run(cmd, capture_output=True, text=True, env=dict(os.environ, RANK="1"), timeout=600,
                          cwd=ROOT)
    assert out1.returncode == 0 and out1.stdout.strip() == ""
