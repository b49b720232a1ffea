"""Writes ``long_pair_1mbp.json``: the oracle's global score and divide-and-conquer
CIGAR of the 1 Mbp x 1 Mbp long pair (seeded generator ``synth.long_pair()``,
global affine +2/-3/-5/-2).

Only ``oracle/`` computes the stored values; ``synth/`` draws the letters. The
pair has 1e12 DP cells, so the two oracle calls run as two processes side by
side, each single-threaded: the linear-space score pass of Sec. III-A (score
only, Fig. 1 right) and the Myers-Miller divide-and-conquer traceback (the
linear-space traceback of Sec. III-A, about 2e12 cells). On one core of an
x86 host the oracle relaxes about 0.1 G cells/s in the score pass and 0.13 G
cells/s in the traceback, so this takes about four and a half hours.

Run from the repository root:  python tests/golden/make_long_pair_golden.py
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "long_pair_1mbp.json")
SCORING = dict(match=2, mismatch=-3, gap_open=-5, gap_extend=-2)


def _pair():
    import synth
    return synth.long_pair().pair(0)


def _score(_):
    import oracle
    q, s = _pair()
    t = time.time()
    S, ei, ej = oracle.score(q, s, oracle.Scoring(**SCORING), oracle.GLOBAL)
    return dict(score=S, end=[ei, ej], seconds=round(time.time() - t, 1))


def _cigar(_):
    import oracle
    q, s = _pair()
    t = time.time()
    cig, cells = oracle.hirschberg(q, s, oracle.Scoring(**SCORING))
    return dict(cigar=oracle.cigar_string(cig), cigar_words=int(len(cig)), cells_relaxed=cells,
                base_cells=oracle.BASE_CELLS, seconds=round(time.time() - t, 1))


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=np.uint8).tobytes()).hexdigest()


def main():
    import oracle
    oracle.build()
    q, s = _pair()
    ctx = mp.get_context("spawn")
    with ctx.Pool(2) as pool:
        sc_res = pool.apply_async(_score, (0,))
        cg_res = pool.apply_async(_cigar, (0,))
        a, b = sc_res.get(), cg_res.get()
    rec = {
        "what": "oracle global score and Myers-Miller CIGAR of the 1 Mbp long pair",
        "generator": "synth.long_pair() (seed 4, 1,000,000 letters, 1 % substitutions, "
                     "0.1 % indels of Geometric(0.3) length, two 10 kbp reverse complements)",
        "scoring": SCORING,
        "mode": "global",
        "n": int(len(q)), "m": int(len(s)),
        "q_sha256": digest(q), "s_sha256": digest(s),
        "score": a["score"], "end": a["end"],
        "cigar_words": b["cigar_words"], "cells_relaxed": b["cells_relaxed"],
        "base_cells": b["base_cells"],
        "oracle_seconds": {"score": a["seconds"], "cigar": b["seconds"]},
        "cigar": b["cigar"],
    }
    with open(OUT + ".tmp", "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    os.replace(OUT + ".tmp", OUT)
    print(json.dumps({k: v for k, v in rec.items() if k != "cigar"}))


if __name__ == "__main__":
    main()
