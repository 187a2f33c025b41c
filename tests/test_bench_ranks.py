"""Host logic of the multi-GPU benchmark run, on CPU with gloo at world size 2.

Every rank times its own copy of the workload; the job's time is the slowest
rank's (one all-reduce MAX, the run's only collective) and the value counts
all ranks' vertices.  The reference arm runs on rank 0 only.
"""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 1.5 + rank            # rank 1 is the slowest
        t = bench.slowest_rank_time(mine, device="cpu")
        v = bench.job_value(1_000_000, world, 4, t)
        dist.barrier()
        out[rank] = (t, v)
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_job_time():
    world = 2
    port = 29500 + (os.getpid() % 2000)
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, v = res[rank]
        assert t == 2.5
        assert v == pytest.approx(2 * 1_000_000 * 4 / 2.5 / 1e6)


def test_single_process_needs_no_process_group():
    assert bench.slowest_rank_time(3.0) == 3.0
    assert bench.job_value(10**6, 1, 2, 1.0) == pytest.approx(2.0)


def _run_reference(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--gpus", "2", "--grid", "64", "--tile", "16", "--c", "8",
                           "--cpu-budget", "0.2", "--steps", "2", "--warmup", "3"],
                          capture_output=True, text=True, env=env, timeout=300, cwd=ROOT)


def test_reference_arm_runs_on_rank0_only():
    r1 = _run_reference(1)
    assert r1.returncode == 0, r1.stderr
    assert r1.stdout.strip() == ""
    r0 = _run_reference(0)
    assert r0.returncode == 0, r0.stderr
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
