"""The multi-rank path of bench.py on CPU (gloo, world size 2): one seeded disk per rank, the
slowest rank's times taken by an all-reduce MAX, the whole-job rate from them, and the
reference arm printing from rank 0 alone. The GPU launch itself (NCCL, one rank per GPU) runs
the same functions."""

import json
import os
import socket
import subprocess
import sys

import pytest

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


WORKER = r"""
import json, os, sys
sys.path.insert(0, {repo!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="env://")
rank, world, _ = bench.dist_env()
times = [1.0 + rank, 10.0 - 3.0 * rank, 0.5 * (rank + 1)]
t = bench.rank_max(times, "cpu")
p = bench.workload(rank)
rate = bench.job_rate(p.evals, world, t[0])
print(json.dumps({{"rank": rank, "world": world, "max": t, "rate": rate, "seed": p.seed,
                  "T0": float(p.T.flat[0])}}), flush=True)
dist.destroy_process_group()
"""


def _launch(code, world=2):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=REPO,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for pr in procs:
        out, err = pr.communicate(timeout=240)
        assert pr.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_rank_max_and_job_rate_with_two_gloo_ranks():
    outs = _launch(WORKER.format(repo=REPO))
    res = sorted((json.loads(o.strip().splitlines()[-1]) for o in outs), key=lambda d: d["rank"])
    for d in res:
        assert d["world"] == 2
        assert d["max"] == [2.0, 10.0, 1.0]       # element-wise max over the ranks
        from paper_2509_03623_b300 import synth
        evals = synth.config_observation(0).evals
        assert d["rate"] == pytest.approx(evals * 2 / (2.0e-3) / 1e9)
    assert res[0]["seed"] != res[1]["seed"] and res[0]["T0"] != res[1]["T0"]  # own disks


def test_reference_arm_prints_from_rank_zero_only():
    """--impl reference under two ranks: rank 0 times the oracle and prints one JSON line,
    rank 1 exits 0 without output."""
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen(
            [sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
             "--warmup", "3", "--cpu-budget", "1"], env=env, cwd=REPO, stdout=subprocess.PIPE,
            stderr=subprocess.PIPE, text=True))
    outs = []
    for pr in procs:
        out, err = pr.communicate(timeout=600)
        assert pr.returncode == 0, err[-2000:]
        outs.append(out.strip())
    assert outs[1] == ""
    d = json.loads(outs[0].splitlines()[-1])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
