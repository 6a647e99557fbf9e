"""The multi-process path of bench.py on CPU (world size 2, gloo): every rank
runs its own replica, the timing collectives take the slowest rank, the
whole-job value counts every rank's units, and only rank 0 reports."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    reps = bench.Replicas("gloo")
    reps.barrier()
    slowest = reps.max(1.0 + rank)                       # rank 1 takes longer
    value = reps.whole_job(100, 0.5 + 0.25 * rank)       # 100 units per rank
    q.put((rank, reps.ws, slowest, value))
    reps.close()


def test_replicas_take_the_slowest_rank_and_count_every_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ws, slowest, value in got:
        assert ws == 2 and slowest == 2.0
        assert value == pytest.approx(200 / 0.75)          # all units / the slowest rank's seconds


def test_reference_arm_under_torchrun_reports_once():
    """torchrun with two ranks: rank 0 times the oracle and prints one JSON
    line, rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-seconds", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2
    assert lines[0]["value"] > 0 and lines[0]["cpu_baseline"]["kind"] == "oracle"
