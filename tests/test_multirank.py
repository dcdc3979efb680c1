"""Multi-rank paths on CPU (gloo, world size 2): throughput aggregation over
ranks and the reference arm's rank-0-only rule."""
import os
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    local_ms = 1000.0 if rank == 0 else 1500.0       # rank 1 is the slow one
    value, total = bench.combine_ranks(world, 2000, 5, local_ms, reduce_max)
    out[rank] = (value, total)
    dist.destroy_process_group()


def test_weak_scaling_uses_slowest_rank():
    world, port = 2, 29731
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        value, total = out[r]
        assert total == 1500.0
        assert abs(value - world * 2000 * 5 / 1.5) < 1e-9


def test_reference_arm_nonzero_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
