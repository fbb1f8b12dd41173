"""The N > 1 path of the benchmark on CPU: world size 2 over gloo.

Planning runs as independent replicas (one table per GPU, nothing exchanged on the data
path), so what the ranks share is the measurement: barriers, the slowest rank's time and
the whole-job rate. These tests run that logic in two CPU processes, and the benchmark's
reference arm under torchrun, where rank 0 alone measures and prints.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    from paper_2008_03518_gb300.replicas import Replicas

    reps = Replicas("gloo")
    reps.barrier()
    ms = 100.0 * (rank + 1)           # rank 1 is the slow one
    units = 1000 + 10 * rank          # plans this rank scheduled
    rate, slowest = reps.whole_job_rate(units, ms)
    out.put((rank, reps.world, reps.max(rank), slowest, rate))
    reps.barrier()
    reps.close()


def test_two_ranks_share_the_slowest_time_and_the_whole_job_rate():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    for rank, world, mx, slowest, rate in got:
        assert world == 2 and mx == 1.0
        assert slowest == 200.0                       # max over ranks
        assert rate == pytest.approx((1000 + 1010) / 0.2)  # all ranks' plans / slowest time


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    from paper_2008_03518_gb300.replicas import Replicas

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    reps = Replicas("gloo")
    assert reps.world == 1 and reps.max(3.5) == 3.5 and reps.sum(2.0) == 2.0
    rate, ms = reps.whole_job_rate(500, 250.0)
    assert rate == 2000.0 and ms == 250.0


def test_reference_arm_under_torchrun_prints_once_from_rank_zero():
    env = dict(os.environ)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-requests", "1"]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["unit"] == line["unit"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] == 3
