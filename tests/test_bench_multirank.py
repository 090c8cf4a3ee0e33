"""The N > 1 path of bench.py on CPU: two gloo ranks (world size 2, no GPU)
check the max-over-ranks timing and the whole-job throughput, and that the
reference arm does its work on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RANK_SCRIPT = r'''
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
t_local = 1.0 + rank            # rank 1 is the slow one
t = bench.rank_max(dist, t_local, "cpu")
out = {"rank": rank, "t": t, "value": bench.job_throughput(world, 5, t)}
dist.barrier()
print(json.dumps(out), flush=True)
dist.destroy_process_group()
'''


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_over_ranks_and_job_throughput():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r),
                   WORLD_SIZE="2", LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, "-c", _RANK_SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["t"] == 2.0                 # the slowest rank's time on every rank
        assert o["value"] == 2 * 5 / 2.0     # world x steps / that time


def test_reference_arm_other_ranks_do_no_work():
    import bench

    class A:
        warmup, steps, gpus = 1, 1, 2

    assert bench.run_reference(A(), 1, 2) is None  # returns at once: no oracle run on rank 1
