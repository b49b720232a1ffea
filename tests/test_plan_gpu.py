"""GPU tests of graph plans (anyseq_plan_*): a batch shape captured in a CUDA
graph gives, on every replay, the results of anyseq_align_batch on the same
letters (which the oracle pins elsewhere) for new letters of the same shape,
and its letter check still reports a bad code on a replay."""
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


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_plan_replays_match_align_batch_and_oracle(pkg, mode):
    sc_args = (1, -4, -6, -1)
    batches = [synth.random_pairs(700, 0, 330, seed=9100 + k, related=0.7, p_sub=0.05, p_indel=0.02) for k in range(3)]
    # one shape: every batch takes the lengths of the first
    b0 = batches[0]
    shaped = []
    for k, b in enumerate(batches):
        st = synth.Stream(9200 + k, 1)
        q = synth.random_codes(st, len(b0.q), 4)
        s = synth.random_codes(st, len(b0.s), 4)
        if k == 0:
            q, s = b0.q, b0.s
        else:
            q[: len(b.q) // 2] = b.q[: len(b.q) // 2]  # part related, part random
        shaped.append(synth.Batch(q, b0.q_off, s, b0.s_off, 4))
    plan = pkg.Plan(b0.q_off, b0.s_off, pkg.Scoring.make(*sc_args), mode)
    ctx = pkg.Context(0)
    try:
        for b in shaped + shaped[:1]:
            plan.q.copy_(torch.from_numpy(b.q))
            plan.s.copy_(torch.from_numpy(b.s))
            plan.run()
            plan.wait()
            got = plan.results()
            want, _ = ctx.align_batch(b.q, b.q_off, b.s, b.s_off, pkg.Scoring.make(*sc_args), mode)
            assert np.array_equal(got["score"], want["score"])
            assert np.array_equal(got["end_q"], want["end_q"]) and np.array_equal(got["end_s"], want["end_s"])
        idx = np.arange(0, shaped[1].n_pairs, 37)
        sub = shaped[1].subset(idx)
        plan.q.copy_(torch.from_numpy(shaped[1].q)); plan.s.copy_(torch.from_numpy(shaped[1].s))
        plan.run(); plan.wait()
        o = oracle.score_batch(sub, oracle.Scoring(*sc_args), mode)
        assert np.array_equal(plan.results()["score"][idx], o[0])
    finally:
        plan.close()
        ctx.close()


def test_plan_replay_reports_bad_letter(pkg):
    b = synth.random_pairs(200, 10, 120, seed=9300)
    plan = pkg.Plan(b.q_off, b.s_off, pkg.Scoring.make(2, -1, 0, -1), 0)
    try:
        plan.q.copy_(torch.from_numpy(b.q)); plan.s.copy_(torch.from_numpy(b.s))
        plan.run(); plan.wait()     # first run: executed, then captured
        plan.run(); plan.wait()     # replay
        bad = b.q.copy()
        bad[5] = 7
        plan.q.copy_(torch.from_numpy(bad))
        plan.run()
        with pytest.raises(pkg.AnyseqError) as ei:
            plan.wait()
        assert ei.value.status == 2
        plan.q.copy_(torch.from_numpy(b.q))
        plan.run(); plan.wait()     # good letters again
    finally:
        plan.close()


def test_two_plans_alternating_with_upload_and_download(pkg):
    """Two plans of one shape on two streams, each step uploading its letters
    from pinned host memory, replaying and downloading its records (one
    batch's copies overlapping the other's run), give every batch the
    results of anyseq_align_batch and the oracle's scores on a sample."""
    sc_args = (1, -4, -6, -1)
    b0 = synth.random_pairs(900, 0, 300, seed=9300, related=0.7, p_sub=0.05, p_indel=0.02)
    batches = []
    for k in range(6):
        st = synth.Stream(9400 + k, 1)
        q = synth.random_codes(st, len(b0.q), 4)
        s, _ = synth.mutate(q, b0.q_off, 0.05, 0.02, 0.5, 4, st)
        s = np.resize(s, len(b0.s)).astype(np.uint8)  # the subject letters of the shape's lengths
        batches.append(synth.Batch(q, b0.q_off, s, b0.s_off, 4))
    sc = pkg.Scoring.make(*sc_args)
    plans = [pkg.Plan(b0.q_off, b0.s_off, sc, 2), pkg.Plan(b0.q_off, b0.s_off, sc, 2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hq = [pin(b.q) for b in batches]
    hs = [pin(b.s) for b in batches]
    outs = [torch.zeros(b0.n_pairs * 40, dtype=torch.uint8).pin_memory() for _ in batches]
    ctx = pkg.Context(0)
    try:
        for k, b in enumerate(batches):
            i = k & 1
            if k >= 2:
                plans[i].wait(streams[i])
            plans[i].upload(hq[k], hs[k], streams[i])
            plans[i].run(streams[i])
            plans[i].download(outs[k], streams[i])
        for i in range(2):
            plans[i].wait(streams[i])
        for k, b in enumerate(batches):
            got = outs[k].numpy().view(pkg.RESULT_DTYPE)
            want, _ = ctx.align_batch(b.q, b.q_off, b.s, b.s_off, sc, 2)
            assert np.array_equal(got["score"], want["score"]), k
            assert np.array_equal(got["end_q"], want["end_q"]) and np.array_equal(got["end_s"], want["end_s"]), k
        idx = np.arange(0, b0.n_pairs, 29)
        o = oracle.score_batch(batches[3].subset(idx), oracle.Scoring(*sc_args), 2)
        assert np.array_equal(outs[3].numpy().view(pkg.RESULT_DTYPE)["score"][idx], o[0])
    finally:
        for p in plans:
            p.close()
        ctx.close()
