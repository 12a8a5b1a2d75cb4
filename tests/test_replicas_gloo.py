"""The N > 1 path of bench.py (replicas only: every rank solves its own copy of
the workload; there is no data-path collective) on CPU with the gloo backend:
the timed region's duration is the slowest rank's, the whole-job rate counts
every rank's units, and under torchrun the reference arm prints one line from
rank 0 while the other rank exits cleanly."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)      # rank 1 is the slow replica
    out[rank] = (ms, bench.whole_job_rate(1000.0, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_replica_sets_the_time():
    world = 2
    port = 29500 + os.getpid() % 1000
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, rate = out[r]
        assert ms == 15.0
        assert rate == pytest.approx(1000.0 * 2 / 15e-3)


def test_reference_arm_under_torchrun_prints_once():
    port = 30500 + os.getpid() % 1000
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--workload", "tri32_p2"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_captured_apply_traffic_scaling():
    """The ncu-captured level-0 apply traffic (256 x 256 square, p = 3, 523,264
    blocks) is reported for other p = 3 squares scaled by their block count, and
    as null for other mesh families or degrees."""
    sys.path.insert(0, ROOT)
    import bench
    cap = bench.CAPTURED_APPLY
    assert bench.apply_traffic("square", 3, cap["blocks"], "fp64") == cap["fp64"]
    assert bench.apply_traffic("square", 3, 2_095_104, "fp32") == round(cap["fp32"] * 2_095_104 / 523_264)
    assert bench.apply_traffic("cube", 3, 2_095_104, "fp64") is None
    assert bench.apply_traffic("square", 2, 2_095_104, "fp64") is None
