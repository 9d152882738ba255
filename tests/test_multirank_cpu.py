"""The N > 1 bookkeeping of bench.py on CPU: two gloo ranks (world size 2).

The benchmark runs one independent replica per GPU (the path is not sharded;
no data-path collective).  Its only cross-rank steps are a barrier around the
timed region and the max over ranks of the elapsed time; the job's value
counts every rank's passes over its A.  Here two processes on the host form
a gloo group and run exactly those helpers, and the reference arm's rule that
ranks other than 0 exit without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
dist.barrier()
elapsed = bench.reduce_time_max(0.5 + rank, world, "cpu")  # rank 1 is the slow one
value = bench.job_value(4.0e9, 18, world, elapsed)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "world": world, "elapsed": elapsed, "value": value}))
"""


def free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def launch(code, world, extra_env=None):
    port = free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, REPO_ROOT=ROOT, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   WORLD_SIZE=str(world), LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            p.kill()
            raise
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_two_gloo_ranks_take_the_slowest_time_and_count_both_replicas():
    pytest.importorskip("torch")
    outs = [json.loads(o.strip().splitlines()[-1]) for o in launch(WORKER, 2)]
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["world"] == 2
        assert o["elapsed"] == 1.5                      # max over ranks
        assert abs(o["value"] - 4.0 * 18 * 2 / 1.5) < 1e-9  # GB/s: both ranks' passes / the slowest time


def test_reference_arm_other_ranks_exit_without_work():
    """--impl reference: rank 1 of 2 returns before any oracle work and prints nothing."""
    code = ("import os, sys; sys.path.insert(0, os.environ['REPO_ROOT']); sys.argv = ['bench.py', '--impl', "
            "'reference', '--steps', '1', '--warmup', '3']; import bench; bench.main()")
    port = free_port()
    env = dict(os.environ, REPO_ROOT=ROOT, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK="1",
               WORLD_SIZE="2", LOCAL_RANK="1", CUDA_VISIBLE_DEVICES="")
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_time_max(0.25, 1, "cpu") == 0.25
    assert bench.job_value(1e9, 2, 1, 0.5) == 4.0
