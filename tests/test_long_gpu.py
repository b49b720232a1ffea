"""GPU parity of the long-pair path (anyseq_align_long): the anti-diagonal
stripe wavefront (score) and the divide-and-conquer traceback (CIGAR).

* scores equal the oracle's linear-space global score for lengths that span
  one to many 512-row stripes, ragged tails and n != m;
* the CIGAR equals the oracle's Hirschberg (Myers-Miller) CIGAR under the same
  midpoint rule, for small and large base sizes;
* every CIGAR re-scores to the reported score (a property that holds at any
  size), including a 200 kbp pair shaped like the long-genome workload;
* local and semi-global long pairs: score, optimum cell, start cell and CIGAR
  equal the oracle's linear-space alignment word for word;
* local and semi-global inputs whose score could leave the optimum key's
  range are refused.
"""
import numpy as np
import pytest

import oracle
import synth
from brute import rescore_cigar

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2002_04561_gb300 as p
    p.load(build_if_missing=True)
    return p


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0)
    yield c
    c.close()


C4 = (2, -3, -5, -2)


def related(n, m_extra, seed, p_sub=0.05, p_indel=0.01):
    st = synth.Stream(seed, 1)
    q = synth.random_codes(st, n, 4)
    s, _ = synth.mutate(q, np.array([0, n], np.int64), p_sub, p_indel, 0.3, 4, st)
    return q, s[: max(0, len(s) + m_extra)]


@pytest.mark.parametrize("n", [1, 5, 511, 512, 513, 1500, 3000])
def test_long_score_parity(pkg, ctx, n):
    for k, extra in enumerate([0, -3, 7]):
        q, s = related(n, extra, seed=2000 + n + k)
        out, _ = ctx.align_long(q, s, pkg.Scoring.make(*C4))
        assert out["score"][0] == oracle.score(q, s, oracle.Scoring(*C4))[0]


def test_long_score_unrelated_and_skewed(pkg, ctx):
    st = synth.Stream(2100, 1)
    for n, m in [(2000, 700), (700, 2000), (1025, 1), (1, 1025), (4096, 4096)]:
        q = synth.random_codes(st, n, 4)
        s = synth.random_codes(st, m, 4)
        for args in (C4, (2, -1, 0, -1), (1, -4, -6, -1)):
            out, _ = ctx.align_long(q, s, pkg.Scoring.make(*args))
            assert out["score"][0] == oracle.score(q, s, oracle.Scoring(*args))[0], (n, m, args)


def long_cigar(pkg, ctx, q, s, args):
    cap = len(q) + len(s) + 4
    cig = np.zeros(cap, dtype=np.uint32)
    out, used = ctx.align_long(q, s, pkg.Scoring.make(*args), want=pkg.WANT_SCORE | pkg.WANT_CIGAR, cigar=cig)
    return out[0], cig[:used]


@pytest.mark.parametrize("base", [16, 1024, 1 << 16])
def test_hirschberg_cigar_parity(pkg, ctx, base):
    ctx.set_option("hirschberg_base_cells", base)
    try:
        for k, (n, extra) in enumerate([(40, 3), (700, -5), (1300, 11), (2600, 0)]):
            for args in (C4, (2, -1, 0, -1), (3, -2, -4, -3)):
                q, s = related(n, extra, seed=2200 + k)
                res, cig = long_cigar(pkg, ctx, q, s, args)
                want, _ = oracle.hirschberg(q, s, oracle.Scoring(*args), base)
                assert np.array_equal(cig, want), (n, args, oracle.cigar_string(cig)[:60], oracle.cigar_string(want)[:60])
                assert rescore_cigar(cig, q, s, (0, 0), oracle.Scoring(*args))[0] == res["score"]
    finally:
        ctx.set_option("hirschberg_base_cells", 1 << 16)


def test_hirschberg_unrelated_pairs(pkg, ctx):
    st = synth.Stream(2300, 1)
    for n, m in [(900, 300), (300, 900), (1200, 1250)]:
        q = synth.random_codes(st, n, 4)
        s = synth.random_codes(st, m, 4)
        res, cig = long_cigar(pkg, ctx, q, s, C4)
        want, _ = oracle.hirschberg(q, s, oracle.Scoring(*C4))
        assert np.array_equal(cig, want)


def test_long_pair_60kbp_rescores(pkg, ctx):
    """A 60 kbp pair shaped like the long-genome workload (1 % substitutions,
    0.1 % indels, one 10 kbp inversion): the Hirschberg CIGAR re-scores to the
    score of the wavefront pass, which equals the oracle's score."""
    b = synth.long_pair(seed=4, n=60_000, inversion=10_000, n_inversions=1)
    q, s = b.pair(0)
    res, cig = long_cigar(pkg, ctx, q, s, C4)
    assert rescore_cigar(cig, q, s, (0, 0), oracle.Scoring(*C4))[0] == res["score"]
    assert res["score"] == oracle.score(q, s, oracle.Scoring(*C4))[0]


def test_wavefront_wait_limit_reports_timeout(pkg, ctx):
    """A wait limit of one iteration makes a stripe give up on its predecessor:
    the kernel raises its error flag, every stripe returns, the call reports
    ANYSEQ_ERR_TIMEOUT, and the context keeps working afterwards."""
    q, s = related(5000, 0, seed=2400)
    ctx.set_option("spin_limit", 1)
    try:
        with pytest.raises(pkg.AnyseqError) as ei:
            for _ in range(20):  # a stripe that finds its border already published does not wait
                ctx.align_long(q, s, pkg.Scoring.make(*C4))
        assert ei.value.status == 5
    finally:
        ctx.set_option("spin_limit", 1 << 24)
    out, _ = ctx.align_long(q, s, pkg.Scoring.make(*C4))
    assert out["score"][0] == oracle.score(q, s, oracle.Scoring(*C4))[0]


def tied_long_pairs(seed):
    """Long pairs whose local / semi-global optimum sits where ties are likely:
    a repeated block (two equal local alignments at different rows), a query
    longer than its subject (semi-global last column), and motif repeats."""
    st = synth.Stream(seed, 1)
    X = synth.random_codes(st, 700, 4)
    junk = synth.random_codes(st, 900, 4)
    tail = synth.random_codes(st, 1200, 4)
    motif = synth.random_codes(st, 5, 4)
    return [(np.concatenate([X, junk, X]), X), (X, np.concatenate([X, junk, X])),
            (np.concatenate([X, tail]), X), (np.concatenate([tail, X]), X),
            (np.tile(motif, 300), np.tile(motif, 320))]


@pytest.mark.parametrize("mode", [1, 2])
def test_long_local_and_semiglobal_scores(pkg, ctx, mode):
    """Local and semi-global long pairs on the wavefront: score and optimum cell
    equal the oracle's under the tie rule (larger score, smaller i, smaller j)."""
    st = synth.Stream(2500 + mode, 1)
    pairs = [related(n, extra, seed=2600 + n + mode) for n, extra in ((1, 0), (513, 7), (1800, -40), (3000, 11))]
    pairs += [(synth.random_codes(st, 2000, 4), synth.random_codes(st, 700, 4)),
              (synth.random_codes(st, 600, 4), synth.random_codes(st, 2100, 4))]
    pairs += tied_long_pairs(2700 + mode)
    for args in (C4, (1, -4, -6, -1), (2, -1, 0, -1)):
        for q, s in pairs:
            out, _ = ctx.align_long(q, s, pkg.Scoring.make(*args), mode=mode)
            want = oracle.score(q, s, oracle.Scoring(*args), mode)
            got = (int(out["score"][0]), int(out["end_q"][0]), int(out["end_s"][0]))
            assert got == tuple(int(x) for x in want), (len(q), len(s), args, got, want)


def long_cigar_mode(pkg, ctx, q, s, args, mode):
    cap = len(q) + len(s) + 4
    cig = np.zeros(cap, dtype=np.uint32)
    out, used = ctx.align_long(q, s, pkg.Scoring.make(*args), mode=mode, want=pkg.WANT_SCORE | pkg.WANT_CIGAR,
                               cigar=cig)
    r = out[0]
    return int(r["score"]), (int(r["beg_q"]), int(r["beg_s"])), (int(r["end_q"]), int(r["end_s"])), cig[:used]


@pytest.mark.parametrize("base", [256, 1 << 16])
@pytest.mark.parametrize("mode", [1, 2])
def test_long_local_and_semiglobal_cigars(pkg, ctx, mode, base):
    """Traceback of local and semi-global long pairs: the optimum cell, the
    start cell of the anchored reverse wavefront pass (largest start row, then
    column, among the optimal alignments ending there) and the divide-and-
    conquer CIGAR between them equal the oracle's, word for word; the pairs
    include repeated blocks and a mismatch-0 scheme, where starts tie."""
    st = synth.Stream(3100 + mode, 1)
    core = synth.random_codes(st, 1500, 4)
    planted = (np.concatenate([synth.random_codes(st, 700, 4), core, synth.random_codes(st, 300, 4)]),
               np.concatenate([synth.random_codes(st, 1100, 4), core[::-1].copy(), core, synth.random_codes(st, 90, 4)]))
    pairs = [related(n, extra, seed=3200 + n + mode) for n, extra in ((1, 0), (513, 7), (1800, -40), (3000, 11))]
    pairs += [(synth.random_codes(st, 1900, 4), synth.random_codes(st, 600, 4)), planted]
    pairs += tied_long_pairs(3300 + mode)
    ctx.set_option("hirschberg_base_cells", base)
    try:
        for args in (C4, (1, 0, -2, -1), (2, -1, 0, -1)):
            for q, s in pairs:
                got = long_cigar_mode(pkg, ctx, q, s, args, mode)
                S, beg, end, cig = oracle.long_alignment(q, s, oracle.Scoring(*args), mode, base)
                assert got[:3] == (S, beg, end), (len(q), len(s), args, got[:3], (S, beg, end))
                assert np.array_equal(got[3], cig), (len(q), len(s), args)
                if S > 0:
                    assert rescore_cigar(got[3], q, s, beg, oracle.Scoring(*args)) == (S, end[0], end[1])
    finally:
        ctx.set_option("hirschberg_base_cells", 1 << 16)


@pytest.mark.parametrize("mode", [1, 2])
def test_long_local_and_semiglobal_cigar_60kbp(pkg, ctx, mode):
    """A 60 kbp pair of the long-genome shape embedded in unrelated flanks: the
    CIGAR re-scores to the optimum between the reported start and end cells,
    the start satisfies the mode's rule, and score and end equal the oracle's
    linear-space score."""
    b = synth.long_pair(seed=5, n=60_000, inversion=10_000, n_inversions=1)
    q, s = b.pair(0)
    st = synth.Stream(3400, 1)
    q = np.concatenate([synth.random_codes(st, 3000, 4), q])
    s = np.concatenate([s, synth.random_codes(st, 5000, 4)])
    S, beg, end, cig = long_cigar_mode(pkg, ctx, q, s, C4, mode)
    assert (S,) + end == oracle.score(q, s, oracle.Scoring(*C4), mode)
    assert rescore_cigar(cig, q, s, beg, oracle.Scoring(*C4)) == (S, end[0], end[1])
    if mode == 2:
        assert beg[0] == 0 or beg[1] == 0


def test_key_range_is_checked(pkg, ctx):
    """Local and semi-global optima are searched by keys whose score field holds
    values below 2^21: a pair whose best score could reach that (largest match
    score times min(n, m)) is refused with ERR_ARG before any launch; global
    mode has no such limit."""
    st = synth.Stream(3500, 1)
    q = synth.random_codes(st, 21_000, 4)
    big = (100, -100, -5, -2)
    for mode in (1, 2):
        with pytest.raises(pkg.AnyseqError) as ei:
            ctx.align_long(q, q, pkg.Scoring.make(*big), mode=mode)
        assert ei.value.status == 1
        qo = np.array([0, len(q)], np.int64)
        with pytest.raises(pkg.AnyseqError) as ei:
            ctx.align_batch(q, qo, q, qo, pkg.Scoring.make(*big), mode)
        assert ei.value.status == 1
    out, _ = ctx.align_long(q, q, pkg.Scoring.make(*big))
    assert out["score"][0] == 100 * len(q)


@pytest.mark.parametrize("mode", [1, 2])
def test_small_batches_on_the_wavefront_all_modes(pkg, ctx, mode):
    """A batch of a few large pairs (score and optimum cell) takes the wavefront
    in every mode; an empty pair in the batch gets the empty alignment."""
    pairs = tied_long_pairs(2800 + mode)[:3] + [(related(900, 5, seed=2900)[0], np.zeros(0, np.uint8))]
    b = synth.from_pairs(pairs)
    out, _ = ctx.align_batch(b.q, b.q_off, b.s, b.s_off, pkg.Scoring.make(*C4), mode)
    want = oracle.score_batch(b, oracle.Scoring(*C4), mode)
    assert np.array_equal(out["score"], want[0])
    assert np.array_equal(out["end_q"], want[1]) and np.array_equal(out["end_s"], want[2])


@pytest.mark.parametrize("cell", [1, 2])
def test_wavefront_cell_forms_match_oracle(pkg, ctx, cell):
    """Both cell updates of the wavefront's global passes (the three-input
    maximum, picked for launches with many stripes, and the two-step form)
    give the oracle's scores and divide-and-conquer CIGARs on pairs that span
    several stripes."""
    ctx.set_option("wave_cell", cell)
    try:
        for k, (n, extra) in enumerate([(513, 7), (1800, -40), (3000, 11)]):
            q, s = related(n, extra, seed=3600 + k)
            out, _ = ctx.align_long(q, s, pkg.Scoring.make(*C4))
            assert out["score"][0] == oracle.score(q, s, oracle.Scoring(*C4))[0]
            res, cig = long_cigar(pkg, ctx, q, s, C4)
            want, _ = oracle.hirschberg(q, s, oracle.Scoring(*C4))
            assert np.array_equal(cig, want)
    finally:
        ctx.set_option("wave_cell", 0)


@pytest.mark.parametrize("split", [1, 2])
def test_wavefront_split_steps_match_oracle(pkg, ctx, split):
    """The split step of global passes (rows 0-7 of a lane one column ahead of
    rows 8-15: two independent dependency chains per step) and the plain step
    give the oracle's scores and divide-and-conquer CIGARs on pairs of one to
    six 512-row stripes with ragged ends, the query longer or shorter than
    the subject."""
    ctx.set_option("wave_rows", 16)
    ctx.set_option("wave_cell", 1)
    ctx.set_option("wave_split", split)
    try:
        for k, (n, extra) in enumerate([(1, 3), (40, 0), (513, 7), (1800, -40), (3000, 11)]):
            q, s = related(n, extra, seed=3650 + k)
            out, _ = ctx.align_long(q, s, pkg.Scoring.make(*C4))
            assert out["score"][0] == oracle.score(q, s, oracle.Scoring(*C4))[0], (split, n)
            res, cig = long_cigar(pkg, ctx, q, s, C4)
            want, _ = oracle.hirschberg(q, s, oracle.Scoring(*C4))
            assert np.array_equal(cig, want), (split, n)
    finally:
        ctx.set_option("wave_rows", 0)
        ctx.set_option("wave_cell", 0)
        ctx.set_option("wave_split", 0)


@pytest.mark.parametrize("spread", [0, 1])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_wavefront_draw_order_matches_oracle(pkg, ctx, spread, mode):
    """Stripes drawn in plain order and with held-back first draws (the first
    stripes of a launch on distinct SMs) give the oracle's score, optimum
    cell, start cell and linear-space CIGAR, on pairs of 1 to 47 four-row
    stripes."""
    ctx.set_option("wave_spread", spread)
    ctx.set_option("wave_rows", 4)
    try:
        for k, (n, extra) in enumerate([(90, 2), (2500, -17), (6000, 9)]):
            q, s = related(n, extra, seed=4400 + 10 * mode + k)
            cig = np.zeros(len(q) + len(s) + 4, np.uint32)
            out, used = ctx.align_long(q, s, pkg.Scoring.make(*C4), mode=mode,
                                       want=pkg.WANT_SCORE | pkg.WANT_CIGAR, cigar=cig)
            r = out[0]
            got = (int(r["score"]), (int(r["beg_q"]), int(r["beg_s"])), (int(r["end_q"]), int(r["end_s"])))
            S, beg, end, want = oracle.long_alignment(q, s, oracle.Scoring(*C4), mode)
            assert got == (S, beg, end), (spread, mode, n, got, (S, beg, end))
            assert np.array_equal(cig[:used], want), (spread, mode, n)
    finally:
        ctx.set_option("wave_rows", 0)
        ctx.set_option("wave_spread", 1)


PROTEIN = (0, 0, -11, -1)


def protein_pair(n, extra, seed):
    st = synth.Stream(seed, 1)
    q = synth.random_codes(st, n, 20)
    s, _ = synth.mutate(q, np.array([0, n], np.int64), 0.3, 0.03, 0.5, 20, st)
    return q, s[: max(1, len(s) + extra)]


@pytest.mark.parametrize("base", [256, 1 << 16])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_long_protein_pairs_with_matrix(pkg, ctx, mode, base):
    """Long protein pairs (20 letters, a 20 x 20 matrix) on the wavefront's
    matrix path: score, optimum cell, start cell and divide-and-conquer CIGAR
    equal the oracle's linear-space alignment, for pairs of one to six
    stripes; small base cases run the matrix through the base-case kernel."""
    mat = synth.protein_matrix(3)
    sc = pkg.Scoring.make(*PROTEIN, matrix=mat)
    osc = oracle.Scoring(*PROTEIN, matrix=mat)
    ctx.set_option("hirschberg_base_cells", base)
    try:
        for k, (n, extra) in enumerate([(1, 0), (700, 9), (1800, -30), (3000, 5)]):
            q, s = protein_pair(n, extra, 3700 + 10 * mode + k)
            cap = len(q) + len(s) + 4
            cig = np.zeros(cap, dtype=np.uint32)
            out, used = ctx.align_long(q, s, sc, mode=mode, want=pkg.WANT_SCORE | pkg.WANT_CIGAR, cigar=cig)
            r = out[0]
            got = (int(r["score"]), (int(r["beg_q"]), int(r["beg_s"])), (int(r["end_q"]), int(r["end_s"])))
            S, beg, end, want = oracle.long_alignment(q, s, osc, mode, base)
            assert got == (S, beg, end), (n, mode, got, (S, beg, end))
            assert np.array_equal(cig[:used], want), (n, mode)
    finally:
        ctx.set_option("hirschberg_base_cells", 1 << 16)


@pytest.mark.parametrize("rows", [4, 8, 16])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_wavefront_rows_per_lane_match_oracle(pkg, ctx, rows, mode):
    """Every rows-per-lane count of the wavefront's passes (4-row stripes are
    the automatic choice for pairs too small to fill the GPU with taller ones;
    each mode takes the counts it has) gives the oracle's score, cells and
    linear-space CIGAR, on DNA (2-bit letters) and protein (matrix) pairs that
    span one to fifteen stripes with ragged last stripes."""
    mat = synth.protein_matrix(3)
    cases = [(related(n, extra, seed=4100 + 10 * mode + k), C4, None)
             for k, (n, extra) in enumerate([(1, 0), (129, 5), (700, -9), (1800, 13)])]
    cases += [(protein_pair(n, extra, 4200 + 10 * mode + k), PROTEIN, mat)
              for k, (n, extra) in enumerate([(300, 4), (1500, -7)])]
    ctx.set_option("wave_rows", rows)
    try:
        for (q, s), args, m in cases:
            cig = np.zeros(len(q) + len(s) + 4, np.uint32)
            out, used = ctx.align_long(q, s, pkg.Scoring.make(*args, matrix=m), mode=mode,
                                       want=pkg.WANT_SCORE | pkg.WANT_CIGAR, cigar=cig)
            r = out[0]
            got = (int(r["score"]), (int(r["beg_q"]), int(r["beg_s"])), (int(r["end_q"]), int(r["end_s"])))
            S, beg, end, want = oracle.long_alignment(q, s, oracle.Scoring(*args, matrix=m), mode)
            assert got == (S, beg, end), (rows, mode, len(q), got, (S, beg, end))
            assert np.array_equal(cig[:used], want), (rows, mode, len(q))
    finally:
        ctx.set_option("wave_rows", 0)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_matrix_path_equals_row_profiles_on_dna(pkg, ctx, mode):
    """DNA pairs forced through the matrix path (byte letters, shared query
    profiles) give the same score, cells and CIGAR as the 2-bit row-profile
    path."""
    pairs = [related(n, extra, seed=3800 + n) for n, extra in ((513, 7), (2600, -11))] + tied_long_pairs(3810)[:2]
    for q, s in pairs:
        base = long_cigar_mode(pkg, ctx, q, s, C4, mode)
        ctx.set_option("force_matrix_path", 1)
        try:
            forced = long_cigar_mode(pkg, ctx, q, s, C4, mode)
        finally:
            ctx.set_option("force_matrix_path", 0)
        assert base[:3] == forced[:3] and np.array_equal(base[3], forced[3]), (len(q), len(s), mode)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_small_protein_batches_on_the_matrix_wavefront(pkg, ctx, mode):
    """A batch of a few large protein pairs (scores) runs on the wavefront's
    matrix path, one pass per pair side by side; scores and optimum cells
    equal the oracle's, and an empty pair gets the empty alignment."""
    mat = synth.protein_matrix(3)
    pairs = [protein_pair(n, extra, 3900 + 10 * mode + k) for k, (n, extra) in enumerate([(1500, 7), (900, -20), (2100, 3)])]
    pairs.append((pairs[0][0], np.zeros(0, np.uint8)))
    b = synth.from_pairs(pairs, alphabet=20)
    out = np.zeros(b.n_pairs, dtype=pkg.RESULT_DTYPE)
    res, _ = ctx.align_batch(b.q, b.q_off, b.s, b.s_off, pkg.Scoring.make(*PROTEIN, matrix=mat), mode, out=out)
    want = oracle.score_batch(b, oracle.Scoring(*PROTEIN, matrix=mat), mode)
    assert np.array_equal(res["score"], want[0])
    assert np.array_equal(res["end_q"], want[1]) and np.array_equal(res["end_s"], want[2])


@pytest.mark.parametrize("alphabet", [4, 20])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_mixed_batches_split_long_pairs(pkg, ctx, mode, alphabet):
    """A score-only batch of many short pairs and a few long ones: the long
    pairs run on the wavefront, the rest on the batched kernel through its
    pair selection; every score and optimum cell equals the oracle's."""
    st = synth.Stream(4000 + mode + alphabet, 1)
    pairs = []
    for k in range(3000):
        L = int(st.integers(60, 300, 1)[0])
        q = synth.random_codes(st, L, alphabet)
        s, _ = synth.mutate(q, np.array([0, L], np.int64), 0.1, 0.02, 0.5, alphabet, st)
        pairs.append((q, s))
    for k, L in enumerate((5200, 4300, 6100)):
        q = synth.random_codes(st, L, alphabet)
        s, _ = synth.mutate(q, np.array([0, L], np.int64), 0.1, 0.02, 0.5, alphabet, st)
        pairs.insert(700 * k + 11, (q, s))
    b = synth.from_pairs(pairs, alphabet=alphabet)
    if alphabet == 4:
        args, sco = C4, oracle.Scoring(*C4)
        sc = pkg.Scoring.make(*C4)
    else:
        mat = synth.protein_matrix(3)
        sc, sco = pkg.Scoring.make(*PROTEIN, matrix=mat), oracle.Scoring(*PROTEIN, matrix=mat)
    out = np.zeros(b.n_pairs, dtype=pkg.RESULT_DTYPE)
    res, _ = ctx.align_batch(b.q, b.q_off, b.s, b.s_off, sc, mode, out=out)
    want = oracle.score_batch(b, sco, mode)
    bad = np.nonzero((res["score"] != want[0]) | (res["end_q"] != want[1]) | (res["end_s"] != want[2]))[0]
    assert len(bad) == 0, (len(bad), bad[:5])
