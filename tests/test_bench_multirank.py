"""The benchmark's multi-rank logic on CPU with two gloo ranks (the box runs one GPU,
so a multi-GPU run is only exercised here): the timing of a run is the slowest
rank's, the whole-job throughput counts every replica's units, and the reference arm
does its work on rank 0 only."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
ms = 10.0 * (rank + 1)                      # rank 1 is the slow one
m = bench.max_over_ranks(dist, ms, device="cpu")
v = bench.replica_throughput(1000, world, m / 1e3)
print(json.dumps({"rank": rank, "max_ms": m, "value": v}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_max_over_ranks_and_throughput_with_two_gloo_ranks():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["max_ms"] == 20.0                       # the slowest rank's time
        assert o["value"] == pytest.approx(2 * 1000 / 0.020)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    class A:                                             # the arguments run_reference reads
        sample_rays = 8
        steps = 1
        warmup = 0
    bench.run_reference(A(), rank=1, world=2)            # returns at once: no work, no line
    assert capsys.readouterr().out == ""
