"""Parity at the full sizes the benchmark times, on GPU:

* the 1 Mbp x 1 Mbp global affine pair (1e12 cells): the wavefront score and
  the divide-and-conquer CIGAR equal, word for word, the oracle's score and
  Myers-Miller CIGAR stored in tests/golden/long_pair_1mbp.json (written by
  tests/golden/make_long_pair_golden.py, which calls only the oracle); the
  CIGAR also consumes both sequences and re-scores to the score, which the
  allocation-free entry point reproduces;
* the 65,536 learned-band pairs of 1-10 kbp: the banded route's scores equal
  the full DP's on every pair (the certificate is exact), and both equal the
  oracle on every 128th pair (512 pairs, 1.1e10 cells);
* maximum sizes of a batch: 2^21 tiny pairs in one call, and sequences of
  2^21 - 1 letters (the longest a local or semi-global batch accepts) on
  either side of a pair, beside short pairs, every pair against the oracle;
* the longest pair anyseq_align_long accepts on one side (2^23 - 1 letters
  global, 2^21 - 1 local, against 64), score and optimum cell against the
  oracle, and one letter more refused.
"""
import numpy as np
import pytest

import oracle
import synth
from brute import rescore_cigar

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

C4 = (2, -3, -5, -2)


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


def _long_pair_golden():
    import hashlib
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "long_pair_1mbp.json")) as f:
        g = json.load(f)
    digest = lambda a: hashlib.sha256(np.ascontiguousarray(a, dtype=np.uint8).tobytes()).hexdigest()
    return g, digest


def test_long_pair_1mbp_equals_the_oracle(pkg, ctx):
    golden, digest = _long_pair_golden()
    b = synth.long_pair()
    q, s = b.pair(0)
    # the stored values belong to exactly these letters
    assert (digest(q), digest(s)) == (golden["q_sha256"], golden["s_sha256"])
    assert (golden["n"], golden["m"]) == (len(q), len(s))
    sc = pkg.Scoring.make(*C4)
    qd, sd = torch.from_numpy(q).cuda(), torch.from_numpy(s).cuda()
    res, _ = ctx.align_long(qd, sd, sc)
    score = int(res["score"][0])
    cig = np.zeros(len(q) + len(s) + 4, np.uint32)
    r2, used = ctx.align_long(qd, sd, sc, want=pkg.WANT_SCORE | pkg.WANT_CIGAR, cigar=cig)
    assert int(r2["score"][0]) == score
    got, eq, es = rescore_cigar(cig[:used], q, s, (0, 0), oracle.Scoring(*C4))
    assert (got, eq, es) == (score, len(q), len(s))
    assert score == golden["score"]
    assert oracle.cigar_string(cig[:used]) == golden["cigar"]
    assert used == golden["cigar_words"]
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    pkg.align_long_noalloc(qd, sd, sc, out)
    torch.cuda.synchronize()
    assert int(out.item()) == score


def test_band_workload_full_size_scores_equal_full_dp(pkg, ctx):
    sc = pkg.Scoring.make(*C4)
    train = synth.band_pairs(n_pairs=2048, seed=105)
    ctx.band_train(train.q, train.q_off, train.s, train.s_off, sc, epochs=40, lr=1e-3)
    b = synth.band_pairs()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (dev(b.q), dev(b.q_off), dev(b.s), dev(b.s_off))
    full = torch.zeros(b.n_pairs * 40, dtype=torch.uint8, device="cuda")
    band = torch.zeros_like(full)
    ctx.align_batch(*args, sc, pkg.GLOBAL, out=full)
    ctx.align_batch(*args, sc, pkg.GLOBAL, want=pkg.WANT_SCORE | pkg.BAND_LEARNED, out=band)
    fr = full.cpu().numpy().view(pkg.RESULT_DTYPE)
    br = band.cpu().numpy().view(pkg.RESULT_DTYPE)
    assert np.array_equal(fr["score"], br["score"])
    assert ((br["flags"] & pkg.FLAG_BAND_ACCEPTED) != 0).sum() > 1000
    # every 128th pair (512 pairs, about 1e10 cells) against the oracle
    idx = np.arange(0, b.n_pairs, 128)
    want = oracle.score_batch(b.subset(idx), oracle.Scoring(*C4), 0)
    assert np.array_equal(fr["score"][idx], want[0])
    assert np.array_equal(br["score"][idx], want[0])


def _batch_results(pkg, ctx, b, sc_args, mode):
    sc = pkg.Scoring.make(*sc_args)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.zeros(b.n_pairs * 40, dtype=torch.uint8, device="cuda")
    ctx.align_batch(dev(b.q), dev(b.q_off), dev(b.s), dev(b.s_off), sc, mode, out=out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(pkg.RESULT_DTYPE)


def _assert_equal(res, want):
    for k, name in enumerate(("score", "end_q", "end_s")):
        bad = np.nonzero(res[name] != want[k])[0]
        assert len(bad) == 0, f"{len(bad)} pairs differ in {name}; first {int(bad[0])}"


def test_two_million_tiny_pairs(pkg, ctx):
    """2^21 pairs of 0-12 letters in one call: the sort, the work queue and the
    result scatter at that count; every pair equals the oracle in every mode."""
    b = synth.random_pairs(2 ** 21, 0, 12, seed=1500, related=0.6)
    for mode in (0, 1, 2):
        res = _batch_results(pkg, ctx, b, C4, mode)
        _assert_equal(res, oracle.score_batch(b, oracle.Scoring(*C4), mode))


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_sequences_at_the_length_limit(pkg, ctx, mode):
    """A query of 2^21 - 1 letters against 48 and the reverse (one row stripe
    over 2^21 - 1 columns), with 30 short pairs in the same batch."""
    st = synth.Stream(1501 + mode, 1)
    q = synth.random_codes(st, 2 ** 21 - 1, 4)
    s = q[1000:1048].copy()
    pairs = [(q, s), (s, q)]
    pairs += [(synth.random_codes(st, 100, 4), synth.random_codes(st, 120, 4)) for _ in range(30)]
    b = synth.from_pairs(pairs)
    res = _batch_results(pkg, ctx, b, C4, mode)
    want = oracle.score_batch(b, oracle.Scoring(*C4), mode)
    _assert_equal(res, want)
    if mode != 0:
        assert res["score"][0] == 2 * 48 and res["score"][1] == 2 * 48


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("long_side", ["query", "subject"])
def test_align_long_at_the_length_limit(pkg, ctx, mode, long_side):
    """The longest sequence anyseq_align_long takes (global: 2^23 - 1 letters;
    local: 2^21 - 1, the optimum key's field) against a 64-letter piece of it:
    thousands of row stripes (long query), or one stripe over all the columns
    (long subject). One letter more is refused with ERR_ARG."""
    limit = 2 ** 23 if mode == 0 else 2 ** 21
    st = synth.Stream(1600 + mode, 1)
    big = synth.random_codes(st, limit, 4)
    piece = big[70000:70064].copy()
    sc = pkg.Scoring.make(*C4)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    longest = big[: limit - 1]
    q, s = (longest, piece) if long_side == "query" else (piece, longest)
    r, _ = ctx.align_long(dev(q), dev(s), sc, mode=mode)
    want = oracle.score_batch(synth.from_pairs([(q, s)]), oracle.Scoring(*C4), mode)
    got = (int(r["score"][0]), int(r["end_q"][0]), int(r["end_s"][0]))
    assert got == (int(want[0][0]), int(want[1][0]), int(want[2][0]))
    if mode == 1:
        assert got[0] == 2 * 64
    q, s = (big, piece) if long_side == "query" else (piece, big)
    with pytest.raises(pkg.AnyseqError) as ei:
        ctx.align_long(dev(q), dev(s), sc, mode=mode)
    assert ei.value.status == 1
