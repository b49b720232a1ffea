"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* brute-force enumeration of every alignment for short sequences (all modes,
  linear and affine gaps, match/mismatch and an asymmetric matrix);
* textbook worked examples (tests/golden/textbook.json, each cited);
* special cases that reduce to textbook quantities: Levenshtein distance and
  longest common subsequence;
* invariants: self-alignment, local >= 0, swap symmetry with a transposed
  matrix, empty-sequence closed forms, every CIGAR re-scores to its score;
* the divide-and-conquer traceback re-scores to the full-DP optimum and relaxes
  at most about twice the cells (Sec. III-A).
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from brute import best_global, best_local, best_semiglobal, cigar_ops, rescore_cigar

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "textbook.json")

SCHEMES = [
    oracle.Scoring(2, -1, 0, -1),        # linear
    oracle.Scoring(1, -4, -6, -1),       # affine, short-read style
    oracle.Scoring(2, -3, -5, -2),       # affine, long-pair style
    oracle.Scoring(3, -1, -2, -1),
]


def asym_matrix(seed=21, alphabet=4):
    st = synth.Stream(seed, 1)
    return st.integers(-4, 5, alphabet * alphabet).reshape(alphabet, alphabet).astype(np.int8)


def tiny_pairs(count, lo, hi, seed, alphabet=4):
    st = synth.Stream(seed, 2)
    out = []
    for _ in range(count):
        n, m = st.integers(lo, hi, 2)
        out.append((synth.random_codes(st, int(n), alphabet), synth.random_codes(st, int(m), alphabet)))
    return out


@pytest.mark.parametrize("sc", SCHEMES + [oracle.Scoring(0, 0, -3, -1, matrix=asym_matrix())])
def test_brute_force_global(sc):
    for q, s in tiny_pairs(40, 0, 5, seed=1):
        assert oracle.score(q, s, sc, oracle.GLOBAL)[0] == best_global(q, s, sc)
        assert oracle.align(q, s, sc, oracle.GLOBAL)[0] == best_global(q, s, sc)


@pytest.mark.parametrize("sc", SCHEMES[:3] + [oracle.Scoring(0, 0, -3, -1, matrix=asym_matrix())])
def test_brute_force_local(sc):
    for q, s in tiny_pairs(25, 0, 4, seed=2):
        want = best_local(q, s, sc)
        assert oracle.score(q, s, sc, oracle.LOCAL)[0] == want
        assert oracle.align(q, s, sc, oracle.LOCAL)[0] == want


@pytest.mark.parametrize("sc", SCHEMES[:3] + [oracle.Scoring(0, 0, -3, -1, matrix=asym_matrix())])
def test_brute_force_semiglobal(sc):
    for q, s in tiny_pairs(25, 0, 4, seed=3):
        want = best_semiglobal(q, s, sc)
        assert oracle.score(q, s, sc, oracle.SEMIGLOBAL)[0] == want
        assert oracle.align(q, s, sc, oracle.SEMIGLOBAL)[0] == want


def test_brute_force_longer_global_affine():
    sc = oracle.Scoring(2, -3, -5, -2)
    for q, s in tiny_pairs(4, 6, 7, seed=4):
        assert oracle.score(q, s, sc)[0] == best_global(q, s, sc)


def _golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_textbook_cases(case):
    q = np.array(case["codes_q"], np.uint8) if "codes_q" in case else synth.encode_dna(case["q"])
    s = np.array(case["codes_s"], np.uint8) if "codes_s" in case else synth.encode_dna(case["s"])
    sc = oracle.Scoring(case["match"], case["mismatch"], case["open"], case["extend"])
    mode = oracle.MODES[case["mode"]]
    score, beg, end, cig = oracle.align(q, s, sc, mode)
    assert score == case["score"]
    assert oracle.score(q, s, sc, mode)[0] == case["score"]
    if "cigar" in case:
        assert oracle.cigar_string(cig) == case["cigar"]
        assert list(beg) == case["beg"] and list(end) == case["end"]


DP_TABLES = os.path.join(os.path.dirname(__file__), "golden", "dp_tables.json")


def _dp_tables():
    with open(DP_TABLES) as f:
        return json.load(f)["tables"]


@pytest.mark.parametrize("case", _dp_tables(), ids=lambda c: c["name"])
def test_hand_worked_dp_tables(case):
    """Every cell of a hand-worked global table: H(i, j) is the global score of
    the prefixes q[1..i], s[1..j] (Eqs. 1-5 with the global initialisation)."""
    q, s = synth.encode_dna(case["q"]), synth.encode_dna(case["s"])
    sc = oracle.Scoring(case["match"], case["mismatch"], case["open"], case["extend"])
    for i, row in enumerate(case["H"]):
        for j, h in enumerate(row):
            assert oracle.score(q[:i], s[:j], sc, oracle.GLOBAL)[0] == h, (i, j)


def levenshtein(a, b):
    """Wagner-Fischer unit-cost edit distance (textbook)."""
    prev = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        cur = [i] + [0] * len(b)
        for j in range(1, len(b) + 1):
            cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + (a[i - 1] != b[j - 1]))
        prev = cur
    return prev[-1]


def test_levenshtein_special_case():
    sc = oracle.Scoring(0, -1, 0, -1)
    for q, s in tiny_pairs(30, 0, 40, seed=5):
        assert oracle.score(q, s, sc)[0] == -levenshtein(list(q), list(s))


def test_lcs_special_case_against_brute():
    sc = oracle.Scoring(1, 0, 0, 0)
    for q, s in tiny_pairs(20, 0, 5, seed=6):
        # longest common subsequence by enumerating subsequences of q
        best = 0
        n = len(q)
        for mask in range(1 << n):
            sub = [q[k] for k in range(n) if mask >> k & 1]
            it = iter(list(s))
            if all(any(c == d for d in it) for c in sub):
                best = max(best, len(sub))
        assert oracle.score(q, s, sc)[0] == best


@pytest.mark.parametrize("mode", [oracle.GLOBAL, oracle.LOCAL, oracle.SEMIGLOBAL])
def test_self_alignment(mode):
    st = synth.Stream(7, 1)
    for n in (1, 2, 17, 64, 300):
        q = synth.random_codes(st, n, 4)
        for sc in SCHEMES:
            score, beg, end, cig = oracle.align(q, q, sc, mode)
            assert score == n * sc.match
            assert oracle.cigar_string(cig) == f"{n}M"


def test_local_nonnegative_and_disjoint():
    sc = oracle.Scoring(2, -3, -5, -2)
    st = synth.Stream(8, 1)
    for _ in range(20):
        q = synth.random_codes(st, 30, 2)            # letters 0, 1
        s = synth.random_codes(st, 25, 2) + 2        # letters 2, 3
        assert oracle.score(q, s, sc, oracle.LOCAL) == (0, 0, 0)
    for q, s in tiny_pairs(30, 0, 60, seed=9):
        assert oracle.score(q, s, sc, oracle.LOCAL)[0] >= 0


@pytest.mark.parametrize("mode", [oracle.GLOBAL, oracle.LOCAL, oracle.SEMIGLOBAL])
def test_swap_symmetry_transposed_matrix(mode):
    mat = asym_matrix(seed=31)
    sc = oracle.Scoring(0, 0, -4, -1, matrix=mat)
    sct = oracle.Scoring(0, 0, -4, -1, matrix=mat.T.copy())
    for q, s in tiny_pairs(30, 0, 50, seed=10):
        assert oracle.score(q, s, sc, mode)[0] == oracle.score(s, q, sct, mode)[0]


def test_empty_closed_forms():
    sc = oracle.Scoring(2, -3, -5, -2)
    e = np.zeros(0, np.uint8)
    x = synth.encode_dna("ACGTA")
    assert oracle.align(e, e, sc)[0] == 0
    assert oracle.align(e, x, sc)[0] == -5 - 2 * 5
    assert oracle.cigar_string(oracle.align(e, x, sc)[3]) == "5D"
    assert oracle.align(x, e, sc)[0] == -5 - 2 * 5
    assert oracle.cigar_string(oracle.align(x, e, sc)[3]) == "5I"
    for mode in (oracle.LOCAL, oracle.SEMIGLOBAL):
        assert oracle.score(e, x, sc, mode) == (0, 0, 0)
        assert oracle.score(x, e, sc, mode) == (0, 0, 0)
        assert oracle.align(x, e, sc, mode)[0] == 0


@pytest.mark.parametrize("mode", [oracle.GLOBAL, oracle.LOCAL, oracle.SEMIGLOBAL])
def test_cigar_rescores(mode):
    mat = synth.protein_matrix(seed=3)
    schemes = SCHEMES + [oracle.Scoring(0, 0, -11, -1, matrix=mat, alphabet=20)]
    for k, sc in enumerate(schemes):
        alphabet = sc.alphabet
        b = synth.random_pairs(25, 0, 120, alphabet=alphabet, seed=40 + k)
        for p in range(b.n_pairs):
            q, s = b.pair(p)
            score, beg, end, cig = oracle.align(q, s, sc, mode)
            rs, eq, es = rescore_cigar(cig, q, s, beg, sc)
            assert rs == score
            assert (eq, es) == end
            assert oracle.score(q, s, sc, mode) == (score, end[0], end[1])
            if mode == oracle.GLOBAL:
                assert beg == (0, 0) and end == (len(q), len(s))
            # runs are maximal: no two adjacent words share an op
            assert all((int(a) & 15) != (int(b_) & 15) for a, b_ in zip(cig[:-1], cig[1:]))


def test_batch_matches_single():
    sc = oracle.Scoring(1, -4, -6, -1)
    b = synth.random_pairs(60, 0, 80, seed=50)
    for mode in (oracle.GLOBAL, oracle.LOCAL, oracle.SEMIGLOBAL):
        sco, eq, es = oracle.score_batch(b, sc, mode, threads=3)
        res, cigs = oracle.align_batch(b, sc, mode, threads=3)
        for p in range(b.n_pairs):
            q, s = b.pair(p)
            assert (sco[p], eq[p], es[p]) == oracle.score(q, s, sc, mode)
            assert res[p, 0] == sco[p] and res[p, 3] == eq[p] and res[p, 4] == es[p]
            assert np.array_equal(cigs[p], oracle.align(q, s, sc, mode)[3])


@pytest.mark.parametrize("base", [1, 4, 16, 64, 1 << 16])
def test_hirschberg_rescores_to_optimum(base):
    for k, sc in enumerate(SCHEMES + [oracle.Scoring(1, -1, -1, -1), oracle.Scoring(2, -3, 0, -4)]):
        b = synth.random_pairs(12, 0, 90, seed=60 + k, related=0.6)
        for p in range(b.n_pairs):
            q, s = b.pair(p)
            cig, cells = oracle.hirschberg(q, s, sc, base)
            rs, eq, es = rescore_cigar(cig, q, s, (0, 0), sc)
            assert (eq, es) == (len(q), len(s))
            assert rs == oracle.score(q, s, sc)[0]
            # Sec. III-A: at most about doubling the relaxed cells
            assert cells <= 2 * len(q) * len(s) + base + len(q) + len(s) + 1


def test_hirschberg_with_large_base_is_full_traceback():
    sc = oracle.Scoring(2, -3, -5, -2)
    b = synth.random_pairs(10, 1, 100, seed=70)
    for p in range(b.n_pairs):
        q, s = b.pair(p)
        cig, _ = oracle.hirschberg(q, s, sc, 1 << 20)
        assert np.array_equal(cig, oracle.align(q, s, sc)[3])


def test_last_row_matches_prefix_scores():
    """H(n, j) of the forward pass is the global score of q against s[:j]."""
    sc = oracle.Scoring(2, -3, -5, -2)
    for q, s in tiny_pairs(10, 1, 30, seed=80):
        CC, DD = oracle.last_row(q, s, sc, sc.gap_open)
        for j in range(len(s) + 1):
            assert CC[j] == oracle.score(q, s[:j], sc)[0]
        # the reverse pass is the forward pass of the reversed strings
        RR, SS = oracle.last_row(q, s, sc, sc.gap_open, rev=True)
        R2, S2 = oracle.last_row(q[::-1], s[::-1], sc, sc.gap_open)
        assert np.array_equal(RR, R2) and np.array_equal(SS, S2)


def test_last_row_E_is_best_gap_ending():
    """E(n, j) is the best global score of q vs s[:j] among alignments ending in I."""
    sc = oracle.Scoring(2, -3, -5, -2)
    for q, s in tiny_pairs(10, 1, 5, seed=81):
        CC, DD = oracle.last_row(q, s, sc, sc.gap_open)
        from brute import op_strings, score_ops
        for j in range(1, len(s) + 1):
            cands = [score_ops(o, q, s[:j], sc) for o in op_strings(len(q), j) if o.endswith("I")]
            assert DD[j] == max(cands)


# ---------------------------------------------------------------- start cell of a long-pair traceback
# schemes for the start cell: mismatch 0 makes tied starts common (a mismatch
# before the core costs nothing), and the others make an interior start beat
# every start on the edge of a semi-global matrix
START_SCHEMES = [oracle.Scoring(1, 0, -2, -1), oracle.Scoring(2, -3, -5, -2), oracle.Scoring(1, -4, -6, -1),
                 oracle.Scoring(0, 0, -3, -1, matrix=asym_matrix())]


@pytest.mark.parametrize("mode", [oracle.LOCAL, oracle.SEMIGLOBAL])
@pytest.mark.parametrize("sc", START_SCHEMES)
def test_start_cell_against_brute_force(sc, mode):
    """For every allowed start (i, j) up to the optimum cell, the best global
    score of q[i:ei] against s[j:ej] by enumeration of explicit alignments: its
    maximum is the optimum, and the oracle's start is the largest i, then the
    largest j, reaching it. The CIGAR then re-scores to the optimum from the
    start to the optimum cell."""
    for q, s in tiny_pairs(16, 2, 6, 1200 + mode, alphabet=3):
        S, (bi, bj), (ei, ej), cig = oracle.long_alignment(q, s, sc, mode)
        assert S == (best_local(q, s, sc) if mode == oracle.LOCAL else best_semiglobal(q, s, sc))
        if S == 0:
            assert (bi, bj) == (ei, ej) and len(cig) == 0
            continue
        starts = [(i, j) for i in range(ei + 1) for j in range(ej + 1)
                  if (i, j) != (ei, ej) and (mode == oracle.LOCAL or i == 0 or j == 0)]
        g = {st: best_global(q[st[0]:ei], s[st[1]:ej], sc) for st in starts}
        assert max(g.values()) == S
        assert (bi, bj) == max(st for st in starts if g[st] == S)
        assert rescore_cigar(cig, q, s, (bi, bj), sc) == (S, ei, ej)


def test_start_cell_planted_cases():
    sc = oracle.Scoring(2, -3, -5, -2)
    st = synth.Stream(1300, 1)
    core = synth.random_codes(st, 40, 4)
    # semi-global: q inside s, so the alignment starts in row 0 at the insertion point
    s = np.concatenate([synth.random_codes(st, 17, 4), core, synth.random_codes(st, 9, 4)])
    S, beg, end, cig = oracle.long_alignment(core, s, sc, oracle.SEMIGLOBAL)
    assert (S, beg, end, cigar_ops(cig)) == (80, (0, 17), (40, 57), "M" * 40)
    # local: the planted core between unrelated flanks of A against flanks of C
    q = np.concatenate([np.zeros(12, np.uint8), core, np.zeros(5, np.uint8)])
    s = np.concatenate([np.full(30, 1, np.uint8), core, np.full(7, 1, np.uint8)])
    S, beg, end, cig = oracle.long_alignment(q, s, sc, oracle.LOCAL)
    assert S >= 80 and rescore_cigar(cig, q, s, beg, sc) == (S, end[0], end[1])
    assert beg[0] <= 12 and end[0] >= 52 and beg[1] <= 30 and end[1] >= 70
    # tied local starts (mismatch 0): the later start, without the free mismatch
    sc0 = oracle.Scoring(1, 0, -2, -1)
    S, beg, end, cig = oracle.long_alignment(np.array([0, 1], np.uint8), np.array([2, 1], np.uint8), sc0, oracle.LOCAL)
    assert (S, beg, end, cigar_ops(cig)) == (1, (1, 1), (2, 2), "M")
    # semi-global: the interior start (1, 1) would score 4 (AC against AC), but a
    # start must lie in row 0 or column 0; from (0, 0): T/G mismatch, then AC
    q3, s3 = np.array([3, 0, 1], np.uint8), np.array([2, 0, 1], np.uint8)
    S, beg, end, cig = oracle.long_alignment(q3, s3, sc, oracle.SEMIGLOBAL)
    assert (S, beg, end, cigar_ops(cig)) == (1, (0, 0), (3, 3), "MMM")
    # no positive cell: the empty local alignment at (0, 0)
    S, beg, end, cig = oracle.long_alignment(np.zeros(9, np.uint8), np.full(7, 2, np.uint8), sc, oracle.LOCAL)
    assert (S, beg, end, len(cig)) == (0, (0, 0), (0, 0), 0)


@pytest.mark.parametrize("mode", [oracle.LOCAL, oracle.SEMIGLOBAL])
def test_long_alignment_agrees_with_full_traceback(mode):
    """Same score and optimum cell as the full-matrix traceback, and both CIGARs
    re-score to that score (ties may give different paths)."""
    sc = oracle.Scoring(2, -3, -5, -2)
    for q, s in tiny_pairs(20, 30, 120, 1400 + mode):
        S, beg, end, cig = oracle.long_alignment(q, s, sc, mode, base_cells=64)
        S2, beg2, end2, cig2 = oracle.align(q, s, sc, mode)
        assert (S, end) == (S2, end2)
        assert rescore_cigar(cig, q, s, beg, sc) == (S, end[0], end[1])
        assert rescore_cigar(cig2, q, s, beg2, sc) == (S2, end2[0], end2[1])


def test_long_pair_golden_is_self_consistent():
    """The stored 1 Mbp record (written by tests/golden/make_long_pair_golden.py
    from two separate oracle computations: the linear-space score pass and the
    Myers-Miller traceback, Sec. III-A) belongs to the generator's letters, its
    CIGAR consumes both sequences and re-scores (Eqs. 1-5, affine gaps of
    length L costing open + L * extend) to the stored score, and the traceback
    relaxed at most twice the matrix's cells."""
    import hashlib
    import re
    with open(os.path.join(os.path.dirname(__file__), "golden", "long_pair_1mbp.json")) as f:
        g = json.load(f)
    q, s = synth.long_pair().pair(0)
    digest = lambda a: hashlib.sha256(np.ascontiguousarray(a, dtype=np.uint8).tobytes()).hexdigest()
    assert (digest(q), digest(s)) == (g["q_sha256"], g["s_sha256"])
    assert (g["n"], g["m"]) == (len(q), len(s)) and g["end"] == [len(q), len(s)]
    sc = g["scoring"]
    runs = [(int(k), op) for k, op in re.findall(r"(\d+)([MID])", g["cigar"])]
    assert len(runs) == g["cigar_words"]
    assert "".join(f"{k}{op}" for k, op in runs) == g["cigar"]
    i = j = 0
    score = 0
    for k, op in runs:
        if op == "M":
            same = int(np.count_nonzero(q[i:i + k] == s[j:j + k]))
            score += sc["match"] * same + sc["mismatch"] * (k - same)
            i += k
            j += k
        else:
            score += sc["gap_open"] + k * sc["gap_extend"]
            if op == "I":
                i += k
            else:
                j += k
    assert (i, j) == (len(q), len(s))
    assert score == g["score"]
    assert len(q) * len(s) <= g["cells_relaxed"] <= 2 * len(q) * len(s)
