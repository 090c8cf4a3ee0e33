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


def test_compare_keys_flatten_the_forms():
    """The comparison forms become flat top-level keys of the bench line:
    time, iterations and residual per form (learned: the mean over held-out
    loads and its gains), the batched modes' throughputs; a form that failed
    or is missing adds nothing."""
    import bench

    one = {"time_to_solve_s": 1.5, "iterations": 100, "true_relres": 9e-9}
    forms = {
        "pcg64_csr_jacobi": dict(one),
        "pcg64_mf64_jacobi": {"error": "out of memory"},
        "ir32_64_two_level": dict(one, iterations=345),
        "learned_coarse": {"learned": [dict(one, time_to_solve_s=2.0), dict(one, time_to_solve_s=4.0, iterations=300,
                                                                             true_relres=8e-9)],
                           "iteration_gain": 0.5, "time_gain": 0.25},
        "batch_64x4": {"solves_per_s": 248.0, "fallback_systems": 2, "jacobi": {"solves_per_s": 26.0},
                       "two_level_per_system": {"solves_per_s": 55.0}},
    }
    k = bench.compare_keys(forms)
    assert k["tts_pcg64_csr_jacobi_s"] == 1.5 and k["it_pcg64_csr_jacobi"] == 100
    assert "tts_pcg64_mf64_jacobi_s" not in k and "tts_ir32_64_jacobi_s" not in k
    assert k["it_ir32_64_two_level"] == 345
    assert k["tts_learned_coarse_s"] == 3.0 and k["it_learned_coarse"] == 200
    assert k["relres_learned_coarse"] == 9e-9
    assert k["learned_coarse_iteration_gain"] == 0.5 and k["learned_coarse_time_gain"] == 0.25
    assert k["batch_64x4_solves_per_s"] == 248.0 and k["batch_64x4_fallbacks"] == 2
    assert k["batch_64x4_jacobi_solves_per_s"] == 26.0 and k["batch_64x4_per_system_solves_per_s"] == 55.0
    assert bench.job_throughput(1, 10, 0.5) == 20.0
