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


def test_shard_plan_partitions_and_balances():
    """anyseq_shard_plan (host code of the CUDA library, no GPU needed): for
    every world size the shares are disjoint, cover the batch, differ by at
    most one pair, and their cell counts differ by at most the largest pair."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import synth
    import paper_2002_04561_gb300 as pkg
    pkg.load(build_if_missing=True)
    b = synth.band_pairs(n_pairs=3001, seed=77)  # 1-10 kbp: cell counts spread over two decades
    cells = b.q_len() * b.s_len()
    for world in (1, 2, 3, 4, 7):
        shares = [pkg.shard_plan(b.q_off, b.s_off, world, r) for r in range(world)]
        allidx = np.concatenate(shares)
        assert np.array_equal(np.sort(allidx), np.arange(b.n_pairs))
        assert all(np.all(np.diff(sh) > 0) for sh in shares)
        sizes = [len(sh) for sh in shares]
        assert max(sizes) - min(sizes) <= 1
        load = [int(cells[sh].sum()) for sh in shares]
        assert max(load) - min(load) <= int(cells.max()), (world, load)
    with pytest.raises(pkg.AnyseqError):
        pkg.shard_plan(b.q_off, b.s_off, 2, 2)


SHARD_CHILD = r"""
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import numpy as np
import torch.distributed as dist
import synth
import paper_2002_04561_gb300 as pkg
from paper_2002_04561_gb300 import dist as pdist
dist.init_process_group("gloo")
rank = dist.get_rank()
b = synth.short_reads(n_pairs=1001, seed=7)

def fake_align(q, q_off, s, s_off):
    # host-built records, a pure function of each pair's letters
    n = len(q_off) - 1
    out = np.zeros(n, dtype=pkg.RESULT_DTYPE)
    for p in range(n):
        qa, sa = q[q_off[p]:q_off[p + 1]], s[s_off[p]:s_off[p + 1]]
        out["score"][p] = int(qa.astype(np.int64) @ np.arange(1, len(qa) + 1))
        out["end_q"][p] = len(qa)
        out["end_s"][p] = len(sa)
        out["flags"][p] = rank  # which rank aligned it
    return out

got = pdist.align_batch_sharded(None, b.q, b.q_off, b.s, b.s_off, None, 2, align=fake_align)
if rank == 0:
    want = fake_align(b.q, b.q_off, b.s, b.s_off)
    same = bool(np.array_equal(got["score"], want["score"]) and np.array_equal(got["end_q"], want["end_q"])
                and np.array_equal(got["end_s"], want["end_s"]))
    by_rank = [int((got["flags"] == r).sum()) for r in range(2)]
    print(json.dumps({"rank": 0, "same": same, "by_rank": by_rank}))
else:
    print(json.dumps({"rank": rank, "none": got is None}))
dist.destroy_process_group()
"""


def test_sharded_batch_gathers_records_in_order():
    """One batch split over two gloo ranks by the native partition, each share
    'aligned' by a host-built stand-in, and rank 0 receiving every record in
    the caller's pair order (the gather is the only collective)."""
    pytest.importorskip("torch")
    import json
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", SHARD_CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=180) for p in procs]
    res = []
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
        res.append(json.loads(o.strip().splitlines()[-1]))
    assert res[0]["same"] is True
    assert sorted(res[0]["by_rank"]) == [500, 501]
    assert res[1]["none"] is True
