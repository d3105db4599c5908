"""The N > 1 host path of bench.py on CPU: two gloo ranks (127.0.0.1) take
each timed quantity's maximum over the ranks (a replica job lasts as long as
its slowest rank), and the reference arm runs on rank 0 alone (other ranks
exit 0 without work).  No GPU: the same calls run over NCCL on GPUs."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
r = dist.get_rank()
vals = [1.0 + r, 10.0 - 3.0 * r, 0.25 * r]
out = bench.max_over_ranks(vals, "cpu")
dist.barrier()
print(json.dumps({"rank": r, "world": dist.get_world_size(), "out": out}))
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_over_ranks_two_gloo_ranks():
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    try:
        for p in procs:
            o, e = p.communicate(timeout=120)
            assert p.returncode == 0, e
            outs.append(json.loads(o.strip().splitlines()[-1]))
    finally:
        for p in procs:  # a rank left waiting on its peer is ended here
            if p.poll() is None:
                p.kill()
                p.wait()
    for o in outs:
        assert o["world"] == 2
        assert o["out"] == [2.0, 10.0, 0.25], o


def test_max_over_ranks_single_process_is_identity():
    import bench
    assert bench.max_over_ranks([3.5, 1], "cpu") == [3.5, 1.0]


def test_reference_arm_runs_on_rank_zero_only():
    import bench

    class Args:
        gpus, steps, warmup = 2, 1, 0
    # rank 1 of 2 returns at once: no oracle work, nothing printed
    assert bench.run_reference(Args(), 1, 2) == 0

