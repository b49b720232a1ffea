"""GPU parity of the batched traceback (ANYSEQ_WANT_CIGAR) with the oracle.

Score, optimum cell, start cell and the CIGAR words must be identical to the
oracle's full-matrix traceback under the same tie rules, for all modes, linear
and affine gaps, int16x2 and 32-bit lanes, lengths spanning several 128-row
chunks with ragged tails, and empty sequences. Also: the single 1,000 x 1,100
global pair, buffer-capacity errors, and host/device buffer equivalence.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_align(pkg, ctx, b, sc_args, mode, force32=False, on_device=True):
    sc = pkg.Scoring.make(*sc_args[:4], matrix=sc_args[4] if len(sc_args) > 4 else None)
    cap = int(b.q_len().sum() + b.s_len().sum() + b.n_pairs + 16)
    ctx.set_option("force_int32", int(force32))
    try:
        want = pkg.WANT_SCORE | pkg.WANT_END | pkg.WANT_CIGAR
        if on_device:
            out = torch.zeros(b.n_pairs * 40, dtype=torch.uint8, device="cuda")
            cig = torch.zeros(cap, dtype=torch.int32, device="cuda")
            _, used = ctx.align_batch(dev(b.q), dev(b.q_off), dev(b.s), dev(b.s_off), sc, mode, want=want,
                                      out=out, cigar=cig)
            torch.cuda.synchronize()
            res = out.cpu().numpy().view(pkg.RESULT_DTYPE)
            cig = cig.cpu().numpy().view(np.uint32)
        else:
            cig = np.zeros(cap, dtype=np.uint32)
            res, used = ctx.align_batch(b.q, b.q_off, b.s, b.s_off, sc, mode, want=want, cigar=cig)
    finally:
        ctx.set_option("force_int32", 0)
    cigars = [cig[int(r["cigar_off"]):int(r["cigar_off"]) + int(r["cigar_len"])] for r in res]
    return res, cigars, used


def assert_cigar_parity(b, res, cigars, sc_args, mode):
    sc = oracle.Scoring(*sc_args[:4], matrix=sc_args[4] if len(sc_args) > 4 else None)
    want, wcig = oracle.align_batch(b, sc, mode)
    bad = []
    for p in range(b.n_pairs):
        got = (int(res["score"][p]), int(res["beg_q"][p]), int(res["beg_s"][p]), int(res["end_q"][p]), int(res["end_s"][p]))
        exp = tuple(int(x) for x in want[p])
        if got != exp or not np.array_equal(cigars[p], wcig[p]):
            bad.append(p)
    if bad:
        p = bad[0]
        raise AssertionError(
            f"{len(bad)} of {b.n_pairs} differ; pair {p} n={b.q_len()[p]} m={b.s_len()[p]}: gpu "
            f"{(int(res['score'][p]), int(res['beg_q'][p]), int(res['beg_s'][p]), int(res['end_q'][p]), int(res['end_s'][p]))} "
            f"{oracle.cigar_string(cigars[p])[:80]} vs oracle {tuple(int(x) for x in want[p])} "
            f"{oracle.cigar_string(wcig[p])[:80]}")


SCHEMES = [(2, -1, 0, -1), (1, -4, -6, -1), (2, -3, -5, -2)]


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("sc_args", SCHEMES)
@pytest.mark.parametrize("force32", [False, True])
def test_cigar_parity_random(pkg, ctx, mode, sc_args, force32):
    b = synth.random_pairs(300, 0, 420, seed=900 + mode, related=0.7)
    res, cigars, used = gpu_align(pkg, ctx, b, sc_args, mode, force32=force32)
    assert used == sum(len(c) for c in cigars)
    assert_cigar_parity(b, res, cigars, sc_args, mode)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_cigar_edge_lengths(pkg, ctx, mode):
    st = synth.Stream(910 + mode, 1)
    lengths = [0, 1, 2, 7, 8, 9, 127, 128, 129, 255, 256, 257, 300]
    pairs = [(synth.random_codes(st, n, 4), synth.random_codes(st, m, 4)) for n in lengths for m in lengths[::2]]
    b = synth.from_pairs(pairs)
    for sc_args in SCHEMES:
        res, cigars, _ = gpu_align(pkg, ctx, b, sc_args, mode)
        assert_cigar_parity(b, res, cigars, sc_args, mode)


def test_single_pair_global_linear(pkg, ctx):
    """1,000 x 1,100 uniform ACGT, seed 0, global, +2/-1, gap -2: CIGAR equals the oracle's."""
    b = synth.single_pair()
    args = (2, -1, 0, -2)
    res, cigars, _ = gpu_align(pkg, ctx, b, args, 0)
    assert_cigar_parity(b, res, cigars, args, 0)
    q, s = b.pair(0)
    assert rescore_cigar(cigars[0], q, s, (0, 0), oracle.Scoring(*args))[0] == res["score"][0]


def test_cigar_rescores_large_sample(pkg, ctx):
    """Every GPU CIGAR re-scores to the GPU score (independent of the oracle)."""
    b = synth.short_reads(n_pairs=4096, seed=21)
    args = (1, -4, -6, -1)
    res, cigars, _ = gpu_align(pkg, ctx, b, args, 2)
    sc = oracle.Scoring(*args)
    for p in range(0, b.n_pairs, 7):
        q, s = b.pair(p)
        rs, eq, es = rescore_cigar(cigars[p], q, s, (int(res["beg_q"][p]), int(res["beg_s"][p])), sc)
        assert (rs, eq, es) == (res["score"][p], res["end_q"][p], res["end_s"][p])


def test_host_buffers_and_capacity(pkg, ctx):
    b = synth.random_pairs(50, 1, 200, seed=930)
    sc = pkg.Scoring.make(2, -3, -5, -2)
    want = pkg.WANT_SCORE | pkg.WANT_END | pkg.WANT_CIGAR
    r1, c1, u1 = gpu_align(pkg, ctx, b, (2, -3, -5, -2), 0, on_device=False)
    r2, c2, u2 = gpu_align(pkg, ctx, b, (2, -3, -5, -2), 0, on_device=True)
    assert u1 == u2 and all(np.array_equal(x, y) for x, y in zip(c1, c2))
    small = np.zeros(max(1, u1 - 1), dtype=np.uint32)
    with pytest.raises(pkg.AnyseqError) as ei:
        ctx.align_batch(b.q, b.q_off, b.s, b.s_off, sc, 0, want=want, cigar=small)
    assert ei.value.status == 6


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_cigar_protein_matrix(pkg, ctx, mode):
    mat = synth.protein_matrix(seed=3)
    b = synth.random_pairs(200, 0, 400, alphabet=20, seed=1400 + mode, related=0.7, p_sub=0.3, p_indel=0.03)
    args = (0, 0, -11, -1, mat)
    for force32 in (False, True):
        res, cigars, _ = gpu_align(pkg, ctx, b, args, mode, force32=force32)
        assert_cigar_parity(b, res, cigars, args, mode)


def test_protein_workload_cigar_sampled(pkg, ctx):
    """65,536 protein pairs, Smith-Waterman affine with CIGAR: 1,500-pair sample vs the oracle,
    and every sampled CIGAR re-scores to its score."""
    b = synth.protein_pairs()
    mat = synth.protein_matrix(seed=3)
    args = (0, 0, -11, -1, mat)
    res, cigars, _ = gpu_align(pkg, ctx, b, args, 1)
    st = synth.Stream(1500, 1)
    idx = np.unique(st.integers(0, b.n_pairs - 1, 1500))
    sub = b.subset(idx)
    assert_cigar_parity(sub, res[idx], [cigars[int(p)] for p in idx], args, 1)


@pytest.mark.parametrize("sc_args", [(2, -1, 0, -2), (2, -3, -5, -2), (1, -1, -2, -1)])
def test_small_global_batches_on_the_wavefront(pkg, ctx, sc_args):
    """A few large global pairs run on the wavefront (stripes side by side, its
    own direction-word layout read by the same walk): score, cells and CIGAR
    equal the oracle's full traceback, for the 1,000 x 1,100 pair, related and
    unrelated pairs over several stripes, and a batch holding an empty pair."""
    st = synth.Stream(9400, 1)
    single = synth.single_pair()
    related = []
    for n, extra in ((700, 40), (1300, -25), (2600, 3)):
        q = synth.random_codes(st, n, 4)
        s, _ = synth.mutate(q, np.array([0, n], np.int64), 0.06, 0.02, 0.3, 4, st)
        related.append((q, s[: max(1, len(s) + extra)]))
    unrelated = (synth.random_codes(st, 900, 4), synth.random_codes(st, 1500, 4))
    empty = (synth.random_codes(st, 600, 4), np.zeros(0, np.uint8))
    for b in (single, synth.from_pairs(related), synth.from_pairs([unrelated, empty, related[0]])):
        res, cigars, _ = gpu_align(pkg, ctx, b, sc_args, 0)
        assert_cigar_parity(b, res, cigars, sc_args, 0)


@pytest.mark.parametrize("rows", [4, 8, 16])
def test_wavefront_traceback_rows_per_lane(pkg, ctx, rows):
    """The wavefront's traceback variant at 4, 8 and 16 rows per lane (4-row
    direction words fill the low half of each byte): CIGARs and cells equal
    the oracle's full traceback on small global batches, including pairs of
    one stripe, ragged last stripes and an empty pair."""
    st = synth.Stream(9500 + rows, 1)
    pairs = []
    for n, extra in ((1, 2), (127, 0), (129, 5), (700, -30), (2100, 11)):
        q = synth.random_codes(st, n, 4)
        s, _ = synth.mutate(q, np.array([0, n], np.int64), 0.06, 0.02, 0.3, 4, st)
        pairs.append((q, s[: max(1, len(s) + extra)]))
    pairs.append((synth.random_codes(st, 300, 4), np.zeros(0, np.uint8)))
    ctx.set_option("wave_rows", rows)
    try:
        for sc_args in ((2, -3, -5, -2), (2, -1, 0, -2)):
            # each batch holds a pair above the wavefront's size threshold
            for b in (synth.from_pairs(pairs[:3] + [pairs[4]]), synth.from_pairs(pairs[3:]), synth.single_pair()):
                res, cigars, _ = gpu_align(pkg, ctx, b, sc_args, 0)
                assert_cigar_parity(b, res, cigars, sc_args, 0)
    finally:
        ctx.set_option("wave_rows", 0)


@pytest.mark.parametrize("walker", [1, 2])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_both_walkers_match_oracle(pkg, ctx, mode, walker):
    """The traceback walk as a warp per pair (staged windows) and as a thread
    per pair give the oracle's start cells and CIGARs."""
    b = synth.random_pairs(300, 0, 400, seed=4800 + mode, related=0.7, p_sub=0.05, p_indel=0.02)
    ctx.set_option("tb_walker", walker)
    try:
        res, cigars, used = gpu_align(pkg, ctx, b, (2, -3, -5, -2), mode)
        assert used == sum(len(c) for c in cigars)
        assert_cigar_parity(b, res, cigars, (2, -3, -5, -2), mode)
    finally:
        ctx.set_option("tb_walker", 0)


# query lengths at the edges of a lane's rows and of a chunk (16 lanes x R rows,
# any R up to 16, or 10 for local int16x2 with traceback)
BOUNDARY_LENGTHS = [1, 2, 15, 16, 17, 31, 32, 33, 47, 48, 49, 63, 64, 65, 95, 96, 97, 127, 128, 129, 143, 144,
                    145, 159, 160, 161, 175, 176, 177, 255, 256, 257, 319, 320, 321]


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("force32", [False, True])
def test_cigar_row_counts_at_chunk_boundaries(pkg, ctx, mode, force32):
    """Every rows-per-lane count, odd and even, and one or several chunks: 4 pairs
    per query length, so each work item is planned from one length."""
    st = synth.Stream(1450 + mode, 1)
    pairs = []
    for n in BOUNDARY_LENGTHS:
        for k in range(4):
            q = synth.random_codes(st, n, 4)
            s, _ = synth.mutate(q, np.array([0, n], np.int64), 0.08, 0.02, 0.3, 4, st)
            if k == 3:
                s = synth.random_codes(st, int(st.integers(1, n + 30, 1)[0]), 4)
            pairs.append((q, s))
    b = synth.from_pairs(pairs)
    sc_args = (2, -3, -5, -2)
    res, cigars, _ = gpu_align(pkg, ctx, b, sc_args, mode, force32=force32)
    assert_cigar_parity(b, res, cigars, sc_args, mode)


def _golden_cases():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "textbook.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("force32", [False, True])
def test_golden_cases_on_the_gpu(pkg, ctx, force32):
    """The hand-derived cases of tests/golden/textbook.json (worked examples
    and the tie rules of the optimum cell and the predecessors) through the
    batched path with CIGAR, in int16x2 and in 32-bit lanes: score, cells and
    CIGAR equal the stored hand values, not only the oracle's."""
    for case in _golden_cases():
        q = np.array(case["codes_q"], np.uint8) if "codes_q" in case else synth.encode_dna(case["q"])
        s = np.array(case["codes_s"], np.uint8) if "codes_s" in case else synth.encode_dna(case["s"])
        b = synth.from_pairs([(q, s)])
        args = (case["match"], case["mismatch"], case["open"], case["extend"])
        res, cigars, _ = gpu_align(pkg, ctx, b, args, oracle.MODES[case["mode"]], force32=force32)
        assert int(res["score"][0]) == case["score"], case["name"]
        if "cigar" in case:
            assert oracle.cigar_string(cigars[0]) == case["cigar"], case["name"]
            assert [int(res["beg_q"][0]), int(res["beg_s"][0])] == case["beg"], case["name"]
            assert [int(res["end_q"][0]), int(res["end_s"][0])] == case["end"], case["name"]
