"""bench.py with N > 1: independent replicas, timed by the slowest rank.

Runs two gloo ranks on the CPU (no GPU): the max-over-ranks step time, the
whole-job rate, the per-rank seeds, and the reference arm printing one line
from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [12.5, 20.0][rank]  # rank 1 is the slow one
        job = bench.replica_ms(mine, world)
        out[rank] = (job, bench.job_rate(1000, world, job), bench.replica_seed(7, rank))
    finally:
        tdist.destroy_process_group()


def test_two_ranks_take_the_slowest_step():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(2, free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    assert out[0][0] == out[1][0] == 20.0
    # 2 ranks x 1000 records in 20 ms
    assert out[0][1] == pytest.approx(2 * 1000 / 0.020)
    assert {out[0][2], out[1][2]} == {7, 8}


def test_single_rank_is_unchanged():
    assert bench.replica_ms(3.5, 1) == 3.5
    assert bench.job_rate(10, 1, 1.0) == pytest.approx(10_000.0)


def test_reference_arm_under_torchrun_prints_one_line():
    # the reference arm (the oracle on host cores): rank 0 alone prints
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "1", "--cpu-sample", "20000"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
