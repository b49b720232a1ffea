"""The multi-GPU path of bench.py on CPU: two gloo ranks, as torchrun starts them.

Pairs shard across ranks with no data-path collective; the only collectives are
the timing barrier and the max / sum over ranks, which must combine the ranks'
numbers the way the benchmark reports them (time = slowest rank, work = sum).
The reference arm runs on rank 0 alone; the other ranks exit 0 without work.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
ws, rank, local = bench.dist_env()
dist.init_process_group("gloo")
t = bench.max_over_ranks(ws, 10.0 + rank, "cpu")
w = bench.sum_over_ranks(ws, 100.0 * (rank + 1), "cpu")
bench.barrier(ws)
print(json.dumps({"rank": rank, "max": t, "sum": w, "seed": 2 + 1000 * rank}))
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_combine_like_the_benchmark():
    pytest.importorskip("torch")
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    import json
    res = []
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
        res.append(json.loads(o.strip().splitlines()[-1]))
    assert all(r["max"] == 11.0 for r in res)
    assert all(r["sum"] == 300.0 for r in res)
    assert res[0]["seed"] != res[1]["seed"]  # each rank aligns its own batch


def test_reference_arm_runs_on_rank_zero_only():
    """bench.py --impl reference as two ranks (the launch of an N = 2 run):
    rank 1 exits 0 without work or output, rank 0 prints the reference line."""
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                                       "--gpus", "2", "--steps", "1", "--warmup", "1"],
                                      cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=600) for p in procs]
    import json
    assert procs[1].returncode == 0, outs[1][1]
    assert outs[1][0].strip() == ""
    assert procs[0].returncode == 0, outs[0][1]
    line = json.loads(outs[0][0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
