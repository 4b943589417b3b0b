"""The N > 1 path of bench.py on CPU: two gloo ranks (one process each, as
torchrun would start them) reduce their timings with bench.max_over_ranks and
report the whole job's rate with bench.job_rate.  Replicas only: the data
path has no collective, so the timing reduction is all the ranks share."""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RANK = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
ms = 10.0 + 5.0 * rank                       # this rank's time for 3 steps
t = bench.max_over_ranks(ms, world, "cpu")   # the slowest rank's
rate = bench.job_rate(1000, 3, world, t / 1e3)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "max_ms": t, "rate": rate}))
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_timings():
    pytest.importorskip("torch")
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()),
               WORLD_SIZE="2", REPO_ROOT=ROOT)
    procs = [subprocess.Popen([sys.executable, "-c", _RANK], env=dict(env, RANK=str(r)),
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(2)]
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-2000:]
    res = sorted((json.loads(o.strip().splitlines()[-1]) for o, _ in outs), key=lambda r: r["rank"])
    # both ranks see the slowest rank's 15 ms; 2 ranks x 3 steps x 1000 units
    assert [r["max_ms"] for r in res] == [15.0, 15.0]
    assert res[0]["rate"] == pytest.approx(2 * 3 * 1000 / 0.015 / 1e6)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.job_rate(2_073_600, 20, 1, 0.0112) == pytest.approx(2_073_600 * 20 / 0.0112 / 1e6)
