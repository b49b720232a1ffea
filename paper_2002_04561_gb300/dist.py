"""One batch split over the ranks of a data-parallel job, results gathered.

Pairs are independent (the inter-sequence parallelism of Sec. VI), so a
batch spreads over GPUs with no exchange on the data path: every rank takes
its share from the native partition (``anyseq_shard_plan``: length-balanced
round-robin of the cell-count bins), aligns it on its own GPU, and rank 0
gathers the 40-byte result records and puts them back in the caller's pair
order. The gather is the only collective. This module is argument
marshalling and torch.distributed plumbing; the partition is native and every
alignment step runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np

from . import RESULT_DTYPE, WANT_CIGAR, WANT_END, WANT_SCORE, shard_plan

RECORD_BYTES = RESULT_DTYPE.itemsize


def take_pairs(codes, off, idx):
    """Letters and offsets of the pairs idx (in that order) of one side of a batch."""
    codes = np.asarray(codes)
    off = np.asarray(off, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)
    lens = off[idx + 1] - off[idx]
    new_off = np.zeros(len(idx) + 1, dtype=np.int64)
    np.cumsum(lens, out=new_off[1:])
    if new_off[-1] == 0:
        return np.zeros(0, dtype=codes.dtype), new_off
    # source position of every output letter
    src = np.repeat(off[idx] - new_off[:-1], lens) + np.arange(new_off[-1], dtype=np.int64)
    return np.ascontiguousarray(codes[src]), new_off


def align_batch_sharded(ctx, q, q_off, s, s_off, scoring, mode: int, want: int = WANT_SCORE | WANT_END,
                        group=None, align=None):
    """Align one batch on all ranks of ``group`` (torch.distributed, any
    backend); rank 0 returns every pair's record (RESULT_DTYPE, caller order),
    the other ranks None.

    q, q_off, s, s_off are the whole batch as host arrays, held by every rank
    (each rank copies only its share to its GPU). ``align(q, q_off, s, s_off)``
    aligns one share and returns its records; the default is
    ``ctx.align_batch`` with the given scoring, mode and want. CIGARs are not
    gathered (their words are rank-local), so want must not ask for them.
    """
    import torch
    import torch.distributed as dist

    if want & WANT_CIGAR:
        raise ValueError("align_batch_sharded gathers records only: CIGAR words stay on their rank")
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    q_off = np.ascontiguousarray(q_off, dtype=np.int64)
    s_off = np.ascontiguousarray(s_off, dtype=np.int64)
    n_pairs = len(q_off) - 1
    mine = shard_plan(q_off, s_off, world, rank)
    sq, sq_off = take_pairs(q, q_off, mine)
    ss, ss_off = take_pairs(s, s_off, mine)
    if align is None:
        def align(a, a_off, b, b_off):
            res, _ = ctx.align_batch(a, a_off, b, b_off, scoring, mode, want=want)
            return res
    recs = np.ascontiguousarray(align(sq, sq_off, ss, ss_off)) if len(mine) else np.zeros(0, RESULT_DTYPE)
    if recs.dtype != RESULT_DTYPE or len(recs) != len(mine):
        raise RuntimeError("the share's alignment returned records of the wrong type or count")

    # every rank knows every share's size: pad to the largest and gather raw bytes
    shares = [mine if r == rank else shard_plan(q_off, s_off, world, r) for r in range(world)] if rank == 0 else None
    width = -(-n_pairs // world) * RECORD_BYTES
    device = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    buf = torch.zeros(max(width, 1), dtype=torch.uint8, device=device)
    raw = torch.from_numpy(recs.view(np.uint8).reshape(-1).copy())
    buf[:raw.numel()] = raw.to(device)
    gathered = [torch.zeros_like(buf) for _ in range(world)] if rank == 0 else None
    dst = 0 if group is None else dist.get_global_rank(group, 0)
    dist.gather(buf, gather_list=gathered, dst=dst, group=group)
    if rank != 0:
        return None
    out = np.zeros(n_pairs, dtype=RESULT_DTYPE)
    for r in range(world):
        k = len(shares[r])
        part = gathered[r].cpu().numpy()[:k * RECORD_BYTES].view(RESULT_DTYPE)
        out[shares[r]] = part
    return out
