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
