"""The multi-GPU path of the benchmark (independent replicas, weak scaling)
with world_size-2 gloo process groups on the CPU: disjoint inputs per rank,
the slowest rank's time, the whole-job rate, and the reference arm running
on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import rh_synth  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    try:
        seeds = bench.rank_seeds(rank)
        cube = rh_synth.chromosphere_cube(nx=8, ny=8, ndep=16, seed=seeds["cube"])
        t = bench.max_over_ranks(1.0 + rank, dist)            # rank r "took" 1 + r seconds
        q.put((rank, seeds, float(cube["T"].sum()), t, bench.whole_job_rate(64, ws, 3, t)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, c0, t0, v0), (r1, s1, c1, t1, v1) = res
    # disjoint inputs on each rank, no data exchanged
    assert all(s0[k] != s1[k] for k in s0) and c0 != c1
    # the slowest rank's time on every rank, whole-job rate from it
    assert t0 == t1 == 2.0
    assert v0 == v1 == pytest.approx(2 * 64 * 3 / 2.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
