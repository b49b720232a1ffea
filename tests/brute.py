"""Brute force over explicit alignments: an independent check of the oracle.

Every alignment of two short segments is enumerated as an op string over
M (q_i with s_j), I (q_i against a gap) and D (s_j against a gap) and scored
by summing sigma over M columns and open + k*extend over every maximal run of
I or of D (Sec. III-A's definition of an affine gap of length k). No DP table
is involved, so a mistake in a recurrence, an initialisation or an optimum
rule of the oracle shows up as a different value.
"""
from __future__ import annotations

import itertools


def op_strings(a: int, b: int):
    """All op strings consuming exactly a query and b subject letters."""
    if a == 0 and b == 0:
        yield ""
        return
    if a > 0 and b > 0:
        for rest in op_strings(a - 1, b - 1):
            yield "M" + rest
    if a > 0:
        for rest in op_strings(a - 1, b):
            yield "I" + rest
    if b > 0:
        for rest in op_strings(a, b - 1):
            yield "D" + rest


def score_ops(ops: str, q, s, sc) -> int:
    """Score of an op string aligning q to s from their first letters."""
    total, i, j = 0, 0, 0
    for op, run in itertools.groupby(ops):
        k = len(list(run))
        if op == "M":
            for _ in range(k):
                total += sc.sigma(int(q[i]), int(s[j]))
                i += 1
                j += 1
        elif op == "I":
            total += sc.gap_open + k * sc.gap_extend
            i += k
        else:
            total += sc.gap_open + k * sc.gap_extend
            j += k
    assert i == len(q) and j == len(s)
    return total


def best_global(q, s, sc) -> int:
    return max(score_ops(o, q, s, sc) for o in op_strings(len(q), len(s)))


def best_local(q, s, sc) -> int:
    """Best over every pair of (possibly empty) substrings; the empty alignment scores 0."""
    n, m = len(q), len(s)
    best = 0
    for i0 in range(n + 1):
        for i1 in range(i0, n + 1):
            for j0 in range(m + 1):
                for j1 in range(j0, m + 1):
                    if i1 > i0 or j1 > j0:
                        best = max(best, best_global(q[i0:i1], s[j0:j1], sc))
    return best


def best_semiglobal(q, s, sc) -> int:
    """Free prefix of one sequence (start on row 0 or column 0), free suffix of one
    sequence (end on the last row or the last column)."""
    n, m = len(q), len(s)
    starts = [(i, 0) for i in range(n + 1)] + [(0, j) for j in range(1, m + 1)]
    ends = [(n, j) for j in range(m + 1)] + [(i, m) for i in range(n)]
    best = None
    for i0, j0 in starts:
        for i1, j1 in ends:
            if i1 < i0 or j1 < j0:
                continue
            v = best_global(q[i0:i1], s[j0:j1], sc)
            best = v if best is None else max(best, v)
    return best


def cigar_ops(cigar) -> str:
    return "".join("MID"[int(w) & 15] * (int(w) >> 4) for w in cigar)


def rescore_cigar(cigar, q, s, beg, sc) -> tuple[int, int, int]:
    """Score of a CIGAR placed at DP cell beg; returns (score, end_q, end_s)."""
    ops = cigar_ops(cigar)
    i0, j0 = beg
    nq = ops.count("M") + ops.count("I")
    ns = ops.count("M") + ops.count("D")
    return score_ops(ops, q[i0:i0 + nq], s[j0:j0 + ns], sc), i0 + nq, j0 + ns
