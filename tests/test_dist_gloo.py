"""Multi-rank plumbing of bench.py on CPU: two gloo ranks on 127.0.0.1.

The hot path has no data exchange (replicas only: every rank runs the whole workload on its
own GPU), so what N > 1 adds is host plumbing: the barrier around the timed region, the
maximum of the ranks' times, and one JSON line printed by rank 0.  These tests run that
plumbing with the gloo backend (no GPU).
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    r, ws, local, dist = bench.dist_setup()
    try:
        assert (r, ws, local) == (rank, world, rank)
        assert dist.get_backend() == "gloo"
        bench.barrier(dist)
        q.put((rank, bench.max_over_ranks(dist, 1.5 + 2.0 * rank)))
        bench.barrier(dist)
    finally:
        dist.destroy_process_group()


def test_barrier_and_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 3.5), (1, 3.5)]      # every rank sees the slowest rank's time


def test_single_process_needs_no_process_group(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    sys.path.insert(0, ROOT)
    import bench
    rank, world, local, dist = bench.dist_setup()
    assert (rank, world, local, dist) == (0, 1, 0, None)
    bench.barrier(None)
    assert bench.max_over_ranks(None, 2.25) == 2.25


@pytest.mark.timeout(600)
def test_reference_arm_under_torchrun_two_ranks():
    """`bench.py --impl reference` launched like the multi-GPU bench: rank 0 alone runs the
    oracle and prints one JSON line; rank 1 exits 0 without work."""
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
