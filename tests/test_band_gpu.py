"""GPU tests of the learned band: features, network kernels, exact banded route.

* k-mer diagonal features are bit-identical to the oracle's definition;
* the network's forward outputs and gradients match the float64 reference on
  the same bfloat16 weights (float32 accumulation: relative tolerance 1e-4 on
  outputs and 2e-3 on gradients, i.e. far below the bfloat16 step of 2^-8);
* ANYSEQ_BAND_LEARNED returns exactly the full-DP scores, also for a planted
  band far from the optimal path (the certificate must reject it);
* training on the GPU lowers the loss, and the trained network needs fewer
  banded cells and doublings than the same route without it (a constant band);
* under the shipped defaults the learned route has higher pairs/s than the
  same route with the network's prior (a constant band), all scores equal.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
import synth
from oracle import features as F
from oracle import mlp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

C45 = (2, -3, -5, -2)


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


def test_features_match_oracle(pkg, ctx):
    b = synth.random_pairs(300, 0, 3000, seed=4000, related=0.8, p_sub=0.05, p_indel=0.02)
    got = ctx.band_features(b.q, b.q_off, b.s, b.s_off)
    want = F.features_batch(b)
    assert np.array_equal(got, want)


def test_features_long_query_stride(pkg, ctx):
    st = synth.Stream(4001, 1)
    q = synth.random_codes(st, 40000, 4)
    s, _ = synth.mutate(q, np.array([0, 40000], np.int64), 0.02, 0.002, 0.3, 4, st)
    b = synth.from_pairs([(q, s), (q[:17000], s[:15000])])
    assert np.array_equal(ctx.band_features(b.q, b.q_off, b.s, b.s_off), F.features_batch(b))


def random_params(seed):
    st = synth.Stream(seed, 1)
    params = []
    for a, c in zip(mlp.SIZES[:-1], mlp.SIZES[1:]):
        params.append(((st.uniform(a * c) - 0.5) * 0.4).astype(np.float32).reshape(a, c))
        params.append(((st.uniform(c) - 0.5) * 0.1).astype(np.float32))
    return params


def flat(params):
    return np.concatenate([p.reshape(-1) for p in params]).astype(np.float32)


def bf16_params(params):
    return [mlp.bf16_round(p) if p.ndim == 2 else p for p in params]


def test_forward_and_gradient_match_reference(pkg, ctx):
    params = random_params(4002)
    ctx.band_model_set(flat(params))
    st = synth.Stream(4003, 1)
    B = 777
    x = st.uniform(B * 64).reshape(B, 64).astype(np.float32)
    tgt = np.stack([(st.uniform(B) - 0.5) * 60, np.log(1 + st.uniform(B) * 300)], axis=1).astype(np.float32)
    ref = bf16_params(params)
    y_ref, _ = mlp.forward(ref, x)
    y = ctx.band_forward(x)
    assert np.allclose(y, y_ref, rtol=1e-4, atol=1e-4)
    loss, g = ctx.band_gradient(x, tgt)
    l_ref, g_ref = mlp.grads(ref, x, tgt)
    assert abs(loss - l_ref) <= 1e-4 * max(1.0, abs(l_ref))
    g_ref = np.concatenate([a.reshape(-1) for a in g_ref])
    scale = np.abs(g_ref).max()
    assert np.allclose(g, g_ref, rtol=2e-3, atol=2e-3 * scale)


def test_model_roundtrip(pkg, ctx):
    p = flat(random_params(4004))
    ctx.band_model_set(p)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "band.bin")
        ctx.band_model_save(path)
        ctx.band_model_set(np.zeros_like(p))
        ctx.band_model_load(path)
    assert np.array_equal(ctx.band_model_get(), p)


def constant_model(centre, log_w):
    """A network with constant outputs: centre (columns) and log of the
    half-width relative to the pair's longer sequence."""
    p = np.zeros(25090, np.float32)
    p[-2], p[-1] = centre, log_w
    return p


def band_scores(pkg, ctx, b):
    out, _ = ctx.align_batch(b.q, b.q_off, b.s, b.s_off, pkg.Scoring.make(*C45), pkg.GLOBAL,
                             want=pkg.WANT_SCORE | pkg.BAND_LEARNED)
    return out


def full_scores(pkg, ctx, b):
    out, _ = ctx.align_batch(b.q, b.q_off, b.s, b.s_off, pkg.Scoring.make(*C45), pkg.GLOBAL)
    return out


def band_set(seed, n_pairs=1500):
    return synth.band_pairs(n_pairs=n_pairs, seed=seed, len_lo=300, len_hi=3000)


def test_banded_route_is_exact_and_certificate_rejects_planted_bands(pkg, ctx):
    b = band_set(4005)
    full = full_scores(pkg, ctx, b)
    idx = np.arange(0, b.n_pairs, 11)
    sub = b.subset(idx)
    assert np.array_equal(full["score"][idx], oracle.score_batch(sub, oracle.Scoring(*C45))[0])
    # narrow planted bands (16 to 40 columns at 3 kbp), two of them off the path
    for model in (constant_model(0.0, np.log(0.005)), constant_model(400.0, np.log(0.005)),
                  constant_model(-900.0, np.log(0.013))):
        ctx.band_model_set(model)
        res = band_scores(pkg, ctx, b)
        assert np.array_equal(res["score"], full["score"])
        assert np.array_equal(res["end_q"], b.q_len()) and np.array_equal(res["end_s"], b.s_len())
        accepted = (res["flags"] & pkg.FLAG_BAND_ACCEPTED) != 0
        fallback = (res["flags"] & pkg.FLAG_FULL_FALLBACK) != 0
        assert np.all(accepted ^ fallback)


def test_training_lowers_loss_and_beats_constant_band(pkg, ctx):
    # doublings measure how far a band was from certifying: allow them here, and
    # plan the network's widths as they are (no margin, no floor)
    ctx.set_option("band_max_doublings", 8)
    ctx.set_option("band_area_pct", 50)
    ctx.set_option("band_area16_pct", 50)
    ctx.set_option("band_margin_pct", 100)
    ctx.set_option("band_floor_pct", 0)
    try:
        _training_lowers_loss_and_beats_constant_band(pkg, ctx)
    finally:
        ctx.set_option("band_max_doublings", 0)
        ctx.set_option("band_area_pct", 60)
        ctx.set_option("band_area16_pct", 15)
        ctx.set_option("band_margin_pct", 65)
        ctx.set_option("band_floor_pct", 30)


def _training_lowers_loss_and_beats_constant_band(pkg, ctx):
    train = band_set(105, n_pairs=3000)
    sc = pkg.Scoring.make(*C45)
    ctx.band_model_set(constant_model(0.0, np.log(0.25)))
    first = ctx.band_train(train.q, train.q_off, train.s, train.s_off, sc, epochs=1, lr=1e-3)
    last = ctx.band_train(train.q, train.q_off, train.s, train.s_off, sc, epochs=60, lr=1e-3)
    assert last < first
    test = band_set(4006)
    full = full_scores(pkg, ctx, test)
    res = band_scores(pkg, ctx, test)
    assert np.array_equal(res["score"], full["score"])
    trained_rounds = ctx.stat("band_rounds")
    trained_doublings = int(((res["flags"] >> 8) & 255).sum())
    ctx.band_model_set(constant_model(0.0, np.log(0.005)))
    res0 = band_scores(pkg, ctx, test)
    assert np.array_equal(res0["score"], full["score"])
    const_doublings = int(((res0["flags"] >> 8) & 255).sum())
    assert trained_doublings < const_doublings, (trained_doublings, const_doublings, trained_rounds)


def test_learned_band_gains_over_the_route_without_the_network(pkg):
    """What the trained network gains, under the shipped defaults (no
    doubling, area caps 60/15 %, margin 65 %, floor 30 %): the learned route
    against the same route whose network is replaced by its prior (constant
    outputs: centre 0, half-width a quarter of the longer sequence), on the
    65,536 pairs of the band workload. Both routes' scores equal the full DP
    on every pair; the learned route has the higher pairs/s."""
    import time
    # a fresh context: its network starts from random weights (one trained from a
    # constant model, whose hidden weights are zero, would only move its biases)
    ctx = pkg.Context(0)
    sc = pkg.Scoring.make(*C45)
    train = synth.band_pairs(n_pairs=16384, seed=105)
    ctx.band_train(train.q, train.q_off, train.s, train.s_off, sc, epochs=60, lr=1e-3)
    learned = ctx.band_model_get()
    b = synth.band_pairs()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (dev(b.q), dev(b.q_off), dev(b.s), dev(b.s_off))
    out = torch.zeros(b.n_pairs * 40, dtype=torch.uint8, device="cuda")
    ctx.align_batch(*args, sc, pkg.GLOBAL, out=out)
    full = out.cpu().numpy().view(pkg.RESULT_DTYPE)["score"].copy()

    def route_ms():
        ctx.align_batch(*args, sc, pkg.GLOBAL, want=pkg.WANT_SCORE | pkg.BAND_LEARNED, out=out)
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            ctx.align_batch(*args, sc, pkg.GLOBAL, want=pkg.WANT_SCORE | pkg.BAND_LEARNED, out=out)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        assert np.array_equal(out.cpu().numpy().view(pkg.RESULT_DTYPE)["score"], full)
        return sorted(ts)[1]

    t_learned = route_ms()
    # the route with the network replaced by its prior, a fixed half-width as it is
    ctx.set_option("band_margin_pct", 100)
    ctx.set_option("band_floor_pct", 0)
    ctx.band_model_set(constant_model(0.0, np.log(0.25)))
    t_prior = route_ms()
    ctx.close()
    assert b.n_pairs / t_learned > 1.03 * b.n_pairs / t_prior, (t_learned, t_prior)
