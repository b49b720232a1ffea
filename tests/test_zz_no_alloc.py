"""The allocation-free long-pair score (anyseq_align_long_noalloc).

Callers that cannot let the library allocate device memory (their framework
owns the device memory pool, or they cannot accept the synchronisation of
cudaMalloc/cudaFree) get the global score of a long pair from scratch held in
one fixed device array. This file is collected last, so a run that stops at the
first failure has already run every other test; it also passes on its own.
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


def related(n, seed):
    st = synth.Stream(seed, 1)
    q = synth.random_codes(st, n, 4)
    s, _ = synth.mutate(q, np.array([0, n], np.int64), 0.03, 0.005, 0.3, 4, st)
    return q, s


def test_no_alloc_matches_align_long_on_two_calls(pkg):
    ctx = pkg.Context(0)
    sc = pkg.Scoring.make(2, -3, -5, -2)
    osc = oracle.Scoring(2, -3, -5, -2)
    score = torch.zeros(1, dtype=torch.int32, device="cuda")
    # two calls in a row: the second reuses the array left by the first; the
    # short pair is also scored by the oracle
    for n, seed in [(70_000, 5000), (1_300, 5001)]:
        q, s = related(n, seed)
        dq = torch.from_numpy(q).cuda()
        ds = torch.from_numpy(s).cuda()
        pkg.align_long_noalloc(dq, ds, sc, score)
        want, _ = ctx.align_long(dq, ds, sc)
        assert int(score.item()) == int(want["score"][0])
        if n * len(s) < 10**8:
            assert int(score.item()) == oracle.score(q, s, osc)[0]
    ctx.close()


def test_no_alloc_very_unequal_lengths(pkg):
    """A short query against a long subject and the reverse: the border rows
    follow the subject, the stripe counters the query."""
    ctx = pkg.Context(0)
    sc = pkg.Scoring.make(2, -3, -5, -2)
    osc = oracle.Scoring(2, -3, -5, -2)
    score = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = synth.Stream(5002, 1)
    a = synth.random_codes(st, 300, 4)
    b = synth.random_codes(st, 60_000, 4)
    b[20_000:20_300] = a  # the short sequence sits inside the long one
    for q, s in [(a, b), (b, a)]:
        dq = torch.from_numpy(q).cuda()
        ds = torch.from_numpy(s).cuda()
        pkg.align_long_noalloc(dq, ds, sc, score)
        want, _ = ctx.align_long(dq, ds, sc)
        assert int(score.item()) == int(want["score"][0]) == oracle.score(q, s, osc)[0]
    ctx.close()


def test_no_alloc_rejects_memory_of_another_device(pkg):
    sc = pkg.Scoring.make(2, -3, -5, -2)
    q, s = related(500, 5003)
    score = torch.zeros(1, dtype=torch.int32, device="cuda")
    # host memory is refused before anything runs
    with pytest.raises(pkg.AnyseqError) as ei:
        pkg.align_long_noalloc(torch.from_numpy(q), torch.from_numpy(s), sc, score)
    assert ei.value.status == 1
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU: no memory of another device to pass")
    # q on device 0 but s and the output on device 1
    with pytest.raises(pkg.AnyseqError) as ei:
        pkg.align_long_noalloc(torch.from_numpy(q).cuda(0), torch.from_numpy(s).cuda(1), sc,
                               torch.zeros(1, dtype=torch.int32, device="cuda:1"))
    assert ei.value.status == 1


def test_no_alloc_rejects_oversized_input(pkg):
    sc = pkg.Scoring.make(2, -3, -5, -2)
    score = torch.zeros(1, dtype=torch.int32, device="cuda")
    big = torch.zeros(pkg.NOALLOC_MAX_LEN + 1, dtype=torch.uint8, device="cuda")
    small = torch.zeros(10, dtype=torch.uint8, device="cuda")
    with pytest.raises(pkg.AnyseqError) as ei:
        pkg.align_long_noalloc(big, small, sc, score)
    assert ei.value.status == 1
