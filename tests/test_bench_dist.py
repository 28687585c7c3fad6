"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2).

bench.py runs one replica of the workload per GPU ("replicas only": a single
dense factorisation is not sharded); the ranks meet only at the barrier
around each timed region and at the max over ranks of its time.  These tests
drive those helpers and the launcher contract with CPU processes.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        barrier, max_over_ranks = bench.make_sync(world, torch.device("cpu"))
        barrier()
        t = max_over_ranks(10.0 + rank)  # rank 1 is the slow one
        barrier()
        rate = bench.whole_job_rate(world, 5, 3.0, t)
        out[rank] = (t, rate)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    world = 2
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank_main, args=(world, free_port(), out), nprocs=world, start_method="spawn")
    assert out[0][0] == out[1][0] == 11.0  # both ranks see the slowest time
    # 2 ranks x 5 steps x 3 units in 11 ms
    assert out[0][1] == pytest.approx(2 * 5 * 3.0 / 0.011)


def test_single_rank_helpers_need_no_process_group():
    barrier, max_over_ranks = bench.make_sync(1, torch.device("cpu"))
    barrier()
    assert max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(1, 2, 10.0, 1000.0) == 20.0


def test_reference_arm_under_torchrun_two_ranks():
    # launched the way multi-GPU runs are; rank 0 alone runs the CPU oracle and
    # prints one JSON line, the other rank exits 0 without work
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--ref-sample", "96"]
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
