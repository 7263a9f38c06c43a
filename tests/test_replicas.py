"""The N > 1 bench path on the CPU: two gloo ranks, the whole-job rate of
independent replicas (max of the ranks' times, sum of their work), and the
reference arm's rank handling.  No GPU."""
from __future__ import annotations

import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

from paper_2501_14030_gb300.replicas import job_rate

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took 0.1 (r + 1) s for 1000 (r + 1) units
    t, u, rate = job_rate(0.1 * (rank + 1), 1000.0 * (rank + 1), dist, "cpu")
    dist.barrier()
    out.put((rank, t, u, rate))
    dist.destroy_process_group()


def test_job_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, t, u, rate in res:
        assert t == pytest.approx(0.2) and u == pytest.approx(3000.0)
        assert rate == pytest.approx(3000.0 / 0.2)


def test_job_rate_single_process():
    assert job_rate(0.5, 100.0) == (0.5, 100.0, 200.0)


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference",
                        "--gpus", "2"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
