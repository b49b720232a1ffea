"""GPU parity of the batched path (anyseq_align_batch) with the CPU oracle.

Scores and optimum cells must be bit-identical (integer work). Cases cover all
three modes, linear and affine gaps, match/mismatch and matrix scoring, the
int16x2 lanes and the forced 32-bit lanes, lengths that span several row
chunks (256 rows per chunk) and ragged tails, empty sequences, scorings that
fail the int16 range test, and a 20,000-pair sample of the full 262,144-pair
short-read workload in the launch configuration the benchmark times.
"""
import numpy as np
import pytest

import oracle
import synth

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


def run(pkg, ctx, b, sc_args, mode, on_device=True, force32=False):
    sc = pkg.Scoring.make(*sc_args[:4], matrix=sc_args[4] if len(sc_args) > 4 else None)
    ctx.set_option("force_int32", int(force32))
    try:
        if on_device:
            out = torch.zeros(b.n_pairs * 40, dtype=torch.uint8, device="cuda")
            ctx.align_batch(dev(b.q), dev(b.q_off), dev(b.s), dev(b.s_off), sc, mode, out=out)
            torch.cuda.synchronize()
            return out.cpu().numpy().view(pkg.RESULT_DTYPE)
        out, _ = ctx.align_batch(b.q, b.q_off, b.s, b.s_off, sc, mode)
        return out
    finally:
        ctx.set_option("force_int32", 0)


def oracle_of(b, sc_args, mode):
    sc = oracle.Scoring(*sc_args[:4], matrix=sc_args[4] if len(sc_args) > 4 else None)
    return oracle.score_batch(b, sc, mode)


def assert_parity(res, want, b):
    bad = np.nonzero((res["score"] != want[0]) | (res["end_q"] != want[1]) | (res["end_s"] != want[2]))[0]
    if len(bad):
        p = int(bad[0])
        raise AssertionError(
            f"{len(bad)} of {b.n_pairs} pairs differ; first pair {p} (n={b.q_len()[p]}, m={b.s_len()[p]}): "
            f"gpu ({res['score'][p]}, {res['end_q'][p]}, {res['end_s'][p]}) "
            f"oracle ({want[0][p]}, {want[1][p]}, {want[2][p]})")


SCHEMES = [(2, -1, 0, -1), (1, -4, -6, -1), (2, -3, -5, -2), (3, -2, -4, -3)]
MODES = [0, 1, 2]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("sc_args", SCHEMES)
@pytest.mark.parametrize("force32", [False, True])
def test_random_pairs_parity(pkg, ctx, mode, sc_args, force32):
    b = synth.random_pairs(700, 0, 600, seed=100 + mode, related=0.6)
    res = run(pkg, ctx, b, sc_args, mode, force32=force32)
    assert_parity(res, oracle_of(b, sc_args, mode), b)
    if force32:
        nonempty = (b.q_len() > 0) & (b.s_len() > 0)
        assert np.all(res["flags"][nonempty] & 1)


@pytest.mark.parametrize("mode", MODES)
def test_matrix_scoring_parity(pkg, ctx, mode):
    st = synth.Stream(77, 1)
    mat = st.integers(-5, 6, 16).reshape(4, 4).astype(np.int8)
    b = synth.random_pairs(400, 1, 300, seed=200 + mode)
    args = (0, 0, -4, -1, mat)
    assert_parity(run(pkg, ctx, b, args, mode), oracle_of(b, args, mode), b)


EDGE_LENGTHS = [0, 1, 2, 15, 16, 17, 31, 32, 33, 255, 256, 257, 511, 512, 513, 1000]


@pytest.mark.parametrize("mode", MODES)
def test_edge_lengths(pkg, ctx, mode):
    st = synth.Stream(300 + mode, 1)
    pairs = []
    for n in EDGE_LENGTHS:
        for m in EDGE_LENGTHS:
            if (n * m) % 7 == 0 or n in (0, 1) or m in (0, 1):
                pairs.append((synth.random_codes(st, n, 4), synth.random_codes(st, m, 4)))
    b = synth.from_pairs(pairs)
    for sc_args in SCHEMES[:3]:
        for force32 in (False, True):
            assert_parity(run(pkg, ctx, b, sc_args, mode, force32=force32), oracle_of(b, sc_args, mode), b)


def test_self_alignment_and_identical_pairs(pkg, ctx):
    st = synth.Stream(400, 1)
    pairs = [(x, x) for x in (synth.random_codes(st, int(n), 4) for n in st.integers(1, 700, 100))]
    b = synth.from_pairs(pairs)
    for mode in MODES:
        res = run(pkg, ctx, b, (2, -3, -5, -2), mode)
        assert np.array_equal(res["score"], 2 * b.q_len())


def test_int16_range_test_routes_to_int32(pkg, ctx):
    """Large match scores on long related pairs fail the int16 bound and must be
    computed in 32-bit lanes with exact results."""
    b = synth.random_pairs(200, 500, 900, seed=500, related=1.0, p_sub=0.02, p_indel=0.01)
    args = (40, -40, -40, -5)  # 40 * 500 > 16000: every pair fails the int16 bound
    for mode in MODES:
        res = run(pkg, ctx, b, args, mode)
        assert_parity(res, oracle_of(b, args, mode), b)
        assert np.all(res["flags"] & 1)


def test_host_buffers_match_device_buffers(pkg, ctx):
    b = synth.random_pairs(300, 0, 400, seed=600)
    for mode in MODES:
        a = run(pkg, ctx, b, SCHEMES[1], mode, on_device=True)
        h = run(pkg, ctx, b, SCHEMES[1], mode, on_device=False)
        assert np.array_equal(a["score"], h["score"]) and np.array_equal(a["end_s"], h["end_s"])


@pytest.mark.parametrize("in_place", [0, 1])
def test_pinned_host_letters_read_in_place_or_copied(pkg, ctx, in_place):
    """Host letters in pinned memory, read in place by the packing kernel or
    copied first, give the device-input results and the oracle's, for short
    reads in all three modes (2-bit path) and for a 20-letter batch (always
    copied)."""
    b = synth.random_pairs(3000, 0, 300, seed=710, related=0.7)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    ctx.set_option("host_in_place", in_place)
    try:
        for mode in (0, 1, 2):
            sc = pkg.Scoring.make(2, -3, -5, -2)
            hout = torch.zeros(b.n_pairs * 40, dtype=torch.uint8).pin_memory()
            ctx.align_batch(pin(b.q), pin(b.q_off), pin(b.s), pin(b.s_off), sc, mode, out=hout)
            got = hout.numpy().view(pkg.RESULT_DTYPE)
            dres = run(pkg, ctx, b, (2, -3, -5, -2), mode)
            assert np.array_equal(got["score"], dres["score"]) and np.array_equal(got["end_s"], dres["end_s"])
            want = oracle.score_batch(b, oracle.Scoring(2, -3, -5, -2), mode)
            assert np.array_equal(got["score"], want[0]), mode
        p = synth.random_pairs(500, 20, 200, alphabet=20, seed=711)
        mat = synth.protein_matrix(3)
        hout = torch.zeros(p.n_pairs * 40, dtype=torch.uint8).pin_memory()
        ctx.align_batch(pin(p.q), pin(p.q_off), pin(p.s), pin(p.s_off), pkg.Scoring.make(0, 0, -11, -1, matrix=mat),
                        1, out=hout)
        want = oracle.score_batch(p, oracle.Scoring(0, 0, -11, -1, matrix=mat), 1)
        assert np.array_equal(hout.numpy().view(pkg.RESULT_DTYPE)["score"], want[0])
    finally:
        ctx.set_option("host_in_place", 1)


def test_bad_letter_is_rejected(pkg, ctx):
    b = synth.random_pairs(10, 5, 20, seed=700)
    b.q[3] = 7
    with pytest.raises(pkg.AnyseqError) as ei:
        run(pkg, ctx, b, SCHEMES[0], 0)
    assert ei.value.status == 2


def test_bad_protein_letter_is_rejected(pkg, ctx):
    """A code at or above a 20-letter alphabet, in the query or the subject, on
    the matrix paths (batched score and traceback kernels, and the long-pair
    wavefront): the kernels read a clamped letter (every shared-memory read
    stays inside the profile) and the call fails with ANYSEQ_ERR_ALPHABET;
    the context keeps working."""
    mat = synth.protein_matrix(3)
    sc = pkg.Scoring.make(0, 0, -11, -1, matrix=mat)
    for which, code in (("q", 200), ("s", 255), ("s", 20)):
        b = synth.random_pairs(64, 20, 300, alphabet=20, seed=702)
        getattr(b, which)[157] = code
        for want in (pkg.WANT_SCORE, pkg.WANT_SCORE | pkg.WANT_CIGAR):
            cig = np.zeros(int(b.q_len().sum() + b.s_len().sum() + b.n_pairs), np.uint32)
            with pytest.raises(pkg.AnyseqError) as ei:
                ctx.align_batch(b.q, b.q_off, b.s, b.s_off, sc, 1, want=want, cigar=cig)
            assert ei.value.status == 2, (which, code, want)
    st = synth.Stream(703, 1)
    q = synth.random_codes(st, 3000, 20)
    s = synth.random_codes(st, 2500, 20)
    s[1234] = 240
    for mode in (0, 1, 2):
        with pytest.raises(pkg.AnyseqError) as ei:
            ctx.align_long(q, s, sc, mode=mode)
        assert ei.value.status == 2
    good = synth.random_pairs(16, 20, 100, alphabet=20, seed=704)
    got = run(pkg, ctx, good, (0, 0, -11, -1, mat), 1)
    want = oracle.score_batch(good, oracle.Scoring(0, 0, -11, -1, matrix=mat), 1)
    assert np.array_equal(got["score"], want[0])


def test_bad_arguments_are_rejected(pkg, ctx):
    b = synth.random_pairs(4, 5, 20, seed=701)
    sc = pkg.Scoring.make(1, -1, 2, -1)  # positive open
    with pytest.raises(pkg.AnyseqError) as ei:
        ctx.align_batch(b.q, b.q_off, b.s, b.s_off, sc, 0)
    assert ei.value.status == 1
    with pytest.raises(pkg.AnyseqError):
        ctx.align_batch(b.q, b.q_off, b.s, b.s_off, pkg.Scoring.make(1, -1, 0, -1), 7)
    off = b.q_off.copy()
    off[2], off[3] = off[3], off[2]
    if off[2] > off[3]:
        with pytest.raises(pkg.AnyseqError):
            ctx.align_batch(b.q, off, b.s, b.s_off, pkg.Scoring.make(1, -1, 0, -1), 0)


def test_short_read_workload_full_size_sampled(pkg, ctx):
    """262,144 pairs, semi-global affine +1/-4/-6/-1, int16x2 lanes: every score is
    checked against the oracle on a 20,000-pair sample of the full run."""
    b = synth.short_reads()
    args = (1, -4, -6, -1)
    res = run(pkg, ctx, b, args, 2)
    st = synth.Stream(800, 1)
    idx = np.unique(st.integers(0, b.n_pairs - 1, 20000))
    sub = b.subset(idx)
    want = oracle_of(sub, args, 2)
    assert_parity(res[idx], want, sub)
    assert not np.any(res["flags"] & 1)  # all pairs passed the int16 range test


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("force32", [False, True])
def test_protein_matrix_parity(pkg, ctx, mode, force32):
    """20-letter alphabet with a seeded symmetric matrix (shared-memory query profile path)."""
    mat = synth.protein_matrix(seed=3)
    b = synth.random_pairs(400, 0, 500, alphabet=20, seed=1000 + mode, related=0.7, p_sub=0.3, p_indel=0.03)
    args = (0, 0, -11, -1, mat)
    assert_parity(run(pkg, ctx, b, args, mode, force32=force32), oracle_of(b, args, mode), b)


# query lengths at the edges of a lane's rows and of a chunk: 16 lanes x R rows,
# R up to 16 (row profiles) or 8 (matrix), several chunks above that
BOUNDARY_LENGTHS = [1, 2, 15, 16, 17, 31, 32, 33, 47, 48, 49, 63, 64, 65, 79, 80, 81, 95, 96, 97, 111, 112, 113,
                    127, 128, 129, 143, 144, 145, 175, 176, 177, 255, 256, 257, 383, 384, 385, 511, 512, 513]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("alphabet", [4, 20])
def test_row_counts_at_chunk_boundaries(pkg, ctx, mode, alphabet):
    """Every rows-per-lane count and chunk count: 8 pairs per query length, so each
    4-pair work item is planned from one length (odd and even R, one or several
    chunks; row profiles for 4 letters, the shared-memory matrix profile for 20)."""
    st = synth.Stream(1050 + mode, 1)
    pairs = []
    for n in BOUNDARY_LENGTHS:
        for k in range(8):
            q = synth.random_codes(st, n, alphabet)
            m = int(st.integers(max(1, n - 20), n + 40, 1)[0])
            s = synth.random_codes(st, m, alphabet)
            if k % 2 == 0:   # related pairs: a mutated copy of the query
                s, _ = synth.mutate(q, np.array([0, n], np.int64), 0.1, 0.02, 0.3, alphabet, st)
            pairs.append((q, s))
    b = synth.from_pairs(pairs, alphabet)
    args = (0, 0, -11, -1, synth.protein_matrix(seed=3)) if alphabet == 20 else (2, -3, -5, -2)
    res = run(pkg, ctx, b, args, mode)
    assert_parity(res, oracle_of(b, args, mode), b)
    assert not np.any(res["flags"][(b.q_len() > 0) & (b.s_len() > 0)] & 1)  # int16x2 lanes throughout


def test_wide_alphabet_asymmetric_matrix(pkg, ctx):
    st = synth.Stream(1100, 1)
    mat = st.integers(-6, 9, 32 * 32).reshape(32, 32).astype(np.int8)
    b = synth.random_pairs(200, 1, 300, alphabet=32, seed=1101)
    for mode in MODES:
        args = (0, 0, -7, -2, mat)
        assert_parity(run(pkg, ctx, b, args, mode), oracle_of(b, args, mode), b)


def test_negative_profile_routes_to_int32(pkg, ctx):
    """mismatch below open+extend gives a negative profile byte: 32-bit lanes, exact."""
    b = synth.random_pairs(200, 1, 300, seed=1200)
    args = (2, -10, 0, -1)
    for mode in MODES:
        res = run(pkg, ctx, b, args, mode)
        assert_parity(res, oracle_of(b, args, mode), b)
        nonempty = (b.q_len() > 0) & (b.s_len() > 0)
        assert np.all(res["flags"][nonempty] & 1)


def test_protein_workload_full_size_sampled(pkg, ctx):
    """65,536 protein pairs, local affine (open -11, extend -1): 3,000-pair sample vs the oracle."""
    b = synth.protein_pairs()
    args = (0, 0, -11, -1, synth.protein_matrix(seed=3))
    res = run(pkg, ctx, b, args, 1)
    st = synth.Stream(1300, 1)
    idx = np.unique(st.integers(0, b.n_pairs - 1, 3000))
    sub = b.subset(idx)
    assert_parity(res[idx], oracle_of(sub, args, 1), sub)


def designed_optimum_pairs(seed=7100):
    """Pairs whose optimum sits where the kernel's bookkeeping is most delicate:
    semi-global optima in the last column (query = subject + tail), local
    optima tied between two rows (query = X + junk + X against X) or two
    columns (X against X + junk + X), and motif repeats with many equal
    cells. Lengths vary so the two halves of a lane word differ in length."""
    st = synth.Stream(seed, 1)
    pairs = []
    for k in range(480):
        L = int(st.integers(3, 60, 1)[0])
        X = synth.random_codes(st, L, 4)
        junk = synth.random_codes(st, int(st.integers(0, 90, 1)[0]), 4)
        tail = synth.random_codes(st, int(st.integers(1, 200, 1)[0]), 4)
        kind = k % 6
        if kind == 0:
            pairs.append((np.concatenate([X, tail]), X))
        elif kind == 1:
            pairs.append((np.concatenate([tail, X]), X))
        elif kind == 2:
            pairs.append((np.concatenate([X, junk, X]), X))
        elif kind == 3:
            pairs.append((X, np.concatenate([X, junk, X])))
        elif kind == 4:
            motif = synth.random_codes(st, 3, 4)
            reps = int(st.integers(2, 40, 1)[0])
            pairs.append((np.tile(motif, reps), np.tile(motif, reps + int(st.integers(0, 5, 1)[0]))))
        else:
            pairs.append((np.concatenate([junk, X, tail]), np.concatenate([X, junk[: len(junk) // 2]])))
    return synth.from_pairs(pairs)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("force32", [False, True])
def test_designed_optimum_cells(pkg, ctx, mode, force32):
    b = designed_optimum_pairs()
    for sc_args in SCHEMES + [(1, -1, 0, 0)]:
        assert_parity(run(pkg, ctx, b, sc_args, mode, force32=force32), oracle_of(b, sc_args, mode), b)


@pytest.mark.parametrize("mode", [0, 2])
def test_autotuned_tile_shapes_keep_results(pkg, ctx, mode):
    """The autotuner picks a rows-per-lane cap per length bin from measured SM
    cycles per cell; results with the tuned table equal the untuned ones and the
    oracle's (sampled), and every cap is one of the candidates."""
    b = synth.random_pairs(3000, 10, 600, seed=9600, related=0.7, p_sub=0.05, p_indel=0.02)
    sc_args = (1, -4, -6, -1)
    before = run(pkg, ctx, b, sc_args, mode)
    try:
        caps = ctx.autotune(dev(b.q), dev(b.q_off), dev(b.s), dev(b.s_off), pkg.Scoring.make(*sc_args), mode)
        assert set(np.unique(caps)) <= {0, 4, 8, 12}
        assert ctx.stat("autotune_gain") >= 1.0
        assert ctx.stat("tuned_bins") == int(np.count_nonzero(caps))
        after = run(pkg, ctx, b, sc_args, mode)
        assert np.array_equal(before, after)
        idx = np.arange(0, b.n_pairs, 23)
        assert_parity(after[idx], oracle_of(b.subset(idx), sc_args, mode), b.subset(idx))
    finally:
        ctx.set_option("autotune_reset", 0)


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("cap", [4, 8, 12])
def test_forced_tile_caps_match_oracle(pkg, ctx, mode, cap):
    """Every bin forced to one rows-per-lane cap: queries of 65-128 letters then
    span two or more row chunks of 16 x cap rows (the border scratch must exist
    even though no query is longer than 128), and longer ones many."""
    sc_args = (1, -4, -6, -1)
    try:
        ctx.autotune_set_table(np.full(256, cap, np.uint8))
        for lo, hi, seed in ((65, 128, 9700), (1, 700, 9701)):
            b = synth.random_pairs(700, lo, hi, seed=seed + cap, related=0.7, p_sub=0.05, p_indel=0.02)
            got = run(pkg, ctx, b, sc_args, mode)
            assert_parity(got, oracle_of(b, sc_args, mode), b)
    finally:
        ctx.set_option("autotune_reset", 0)


def test_set_table_rejects_bad_caps(pkg, ctx):
    bad = np.zeros(256, np.uint8)
    bad[17] = 5
    with pytest.raises(pkg.AnyseqError) as ei:
        ctx.autotune_set_table(bad)
    assert ei.value.status == 1
    assert ctx.stat("tuned_bins") == 0
