"""GPU tests of the serving runtime (anyseq_server_*).

* pairs submitted from several threads, of sizes on both sides of the
  long-pair threshold, come back with the oracle's score and optimum cell;
* small pairs are batched (fewer batches than requests), long pairs take the
  wavefront path in every mode (long_pairs statistic);
* admission: a submit beyond the letter budget is refused with ERR_BUDGET and
  queues nothing, and a refused caller can submit again once the server drains;
* a wait with a short limit on an unfinished ticket reports ERR_TIMEOUT and
  keeps the ticket.
"""
import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

C5 = (2, -3, -5, -2)


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2002_04561_gb300 as p
    p.load(build_if_missing=True)
    return p


def mixed_pairs(seed=8100, n=300):
    st = synth.Stream(seed, 1)
    pairs = []
    for k in range(n):
        L = int(st.integers(0, 400, 1)[0]) if k % 25 else int(st.integers(2500, 4000, 1)[0])
        q = synth.random_codes(st, L, 4)
        s, _ = synth.mutate(q, np.array([0, L], np.int64), 0.05, 0.01, 0.3, 4, st)
        pairs.append((q, s))
    return pairs


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_server_results_match_oracle(pkg, mode):
    pairs = mixed_pairs()
    srv = pkg.Server(pkg.Scoring.make(*C5), mode=mode, max_wait_us=300, long_cells=4_000_000)
    try:
        tickets = [None] * len(pairs)

        def producer(lo, hi):
            for k in range(lo, hi):
                tickets[k] = srv.submit(*pairs[k])

        threads = [threading.Thread(target=producer, args=(k * 75, (k + 1) * 75)) for k in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        results = [srv.wait(t) for t in tickets]
        b = synth.from_pairs(pairs)
        want = oracle.score_batch(b, oracle.Scoring(*C5), mode)
        got = np.array([[r["score"], r["end_q"], r["end_s"]] for r, _ in results])
        assert np.array_equal(got[:, 0], want[0])
        assert np.array_equal(got[:, 1], want[1]) and np.array_equal(got[:, 2], want[2])
        assert all(lat > 0 for _, lat in results)
        assert srv.stat("completed") == len(pairs)
        assert srv.stat("batches") < len(pairs)
        n_long = sum(1 for q, s in pairs if len(q) * len(s) >= 4_000_000)
        assert srv.stat("long_pairs") == n_long
        assert srv.stat("held_bytes") == 0
    finally:
        srv.close()


def test_admission_refuses_beyond_budget(pkg):
    st = synth.Stream(8200, 1)
    big = synth.random_codes(st, 3000, 4)
    srv = pkg.Server(pkg.Scoring.make(*C5), mode=0, max_wait_us=200_000, mem_budget=10_000)
    try:
        t1 = srv.submit(big, big)                 # 6,000 letters held
        with pytest.raises(pkg.AnyseqError) as ei:
            srv.submit(big, big)                  # 12,000 > 10,000
        assert ei.value.status == 3
        assert srv.stat("rejected") == 1
        r1, _ = srv.wait(t1)
        assert r1["score"] == 2 * 3000
        t2 = srv.submit(big, big)                 # the budget is free again
        r2, _ = srv.wait(t2)
        assert r2["score"] == 2 * 3000
    finally:
        srv.close()


def test_wait_timeout_keeps_ticket(pkg):
    st = synth.Stream(8300, 1)
    q = synth.random_codes(st, 200, 4)
    # a long batching window: the request is still queued when the short wait expires
    srv = pkg.Server(pkg.Scoring.make(*C5), mode=0, max_wait_us=300_000)
    try:
        t = srv.submit(q, q)
        with pytest.raises(pkg.AnyseqError) as ei:
            srv.wait(t, timeout_us=1000)
        assert ei.value.status == 5
        r, lat = srv.wait(t)
        assert r["score"] == 2 * 200 and lat >= 250_000_000
    finally:
        srv.close()
