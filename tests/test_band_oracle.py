"""Pins of the band oracles (features and network), CPU only.

* features: identical sequences put every hit on the straight line (bin 32);
  a suffix of the query puts every hit on the negative side, with a hit count
  fixed in closed form; a query shifted right by 10 letters puts every hit in
  the hand-computed bin 32 + bucket(10) = 39; the magnitude buckets equal a
  hand-computed table (tests/golden/band_buckets.json); k-mer keys equal a
  per-position recomputation;
* bfloat16 rounding equals torch's float32 -> bfloat16 conversion;
* network gradients equal central finite differences of the loss;
* the first Adam step moves each parameter by -lr * g / (|g| + eps).
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import features as F
from oracle import mlp


def test_kmer_keys_by_direct_recomputation():
    st = synth.Stream(3000, 1)
    q = synth.random_codes(st, 60, 4)
    keys = F.kmer_keys(q)
    for i in range(len(q) - F.K + 1):
        assert keys[i] == sum(int(q[i + t]) << (2 * t) for t in range(F.K))


def test_bucket_table_by_hand():
    with open(os.path.join(os.path.dirname(__file__), "golden", "band_buckets.json")) as f:
        rows = json.load(f)["cases"]
    for x, lg, second, want in rows:
        assert F.bucket(x) == want, x
        if x:
            assert x.bit_length() - 1 == lg  # the table's own arithmetic
            assert want == min(31, 1 + 2 * lg + second)


def test_shifted_copy_hits_one_positive_bin():
    """s = 10 fresh letters + q[:n - 10] (m = n): the query k-mer at i sits at
    j = i + 10, so D = (j - i) * n - (m - n) * i = 10 n, |D| / n = 10, bucket 7
    (floor(log2 10) = 3, second bit 0) and bin 32 + 7 = 39. Sampled starts are
    i = 0, 4, 8, ... (stride 4 below 16,384 letters); the k-mer at i is in s
    when i + 10 + 12 <= n."""
    n = 400
    st = synth.Stream(3003, 1)
    q = synth.random_codes(st, n, 4)
    s = np.concatenate([synth.random_codes(st, 10, 4), q[:n - 10]])
    counts = F.histogram_counts(q, s)
    want = len(range(0, n - 22 + 1, 4))
    assert counts[39] == want and counts.sum() == want


def test_identical_sequences_hit_the_diagonal():
    st = synth.Stream(3001, 1)
    q = synth.random_codes(st, 1000, 4)
    f = F.features(q, q)
    counts = F.histogram_counts(q, q)
    assert counts.sum() == counts[32] >= F.sampled(1000)
    assert f[32] == np.float32(counts[32]) / np.float32(F.sampled(1000)) and f.sum() == f[32]


def test_suffix_hits_are_negative_with_closed_form_count():
    st = synth.Stream(3002, 1)
    n, L = 800, 37
    q = synth.random_codes(st, n, 4)
    s = q[L:]
    counts = F.histogram_counts(q, s)
    assert counts[32:].sum() == 0
    # subject start j matches query start i = j + L, sampled when i % 4 == 0
    expected = sum(1 for j in range(len(s) - F.K + 1) if (j + L) % F.STRIDE == 0)
    assert counts.sum() == expected


def test_short_sequences_have_no_features():
    assert not F.features(np.zeros(5, np.uint8), np.zeros(50, np.uint8)).any()


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    st = synth.Stream(3003, 1)
    x = (st.uniform(5000) - 0.5).astype(np.float32) * np.float32(10.0)
    x[:4] = [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5]
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(mlp.bf16_round(x), want)


def random_params(seed):
    st = synth.Stream(seed, 1)
    params = []
    for a, b in zip(mlp.SIZES[:-1], mlp.SIZES[1:]):
        params.append(mlp.bf16_round(((st.uniform(a * b) - 0.5) * 0.4).astype(np.float32).reshape(a, b)))
        params.append(((st.uniform(b) - 0.5) * 0.1).astype(np.float32))
    return params


def test_gradients_match_finite_differences():
    st = synth.Stream(3004, 1)
    params = [p.astype(np.float64) for p in random_params(3005)]
    x = st.uniform(16 * 64).reshape(16, 64)
    tgt = np.stack([(st.uniform(16) - 0.5) * 40, np.log(1 + st.uniform(16) * 50)], axis=1)
    _, g = mlp.grads(params, x, tgt)
    h = 1e-6
    for k, p in enumerate(params):
        flat = p.reshape(-1)
        for idx in st.integers(0, flat.size - 1, 6):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(params, x, tgt)
            flat[idx] = old - h
            lm = mlp.loss(params, x, tgt)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[idx]) <= 1e-5 * max(1.0, abs(fd)), (k, idx, fd, g[k].reshape(-1)[idx])


def test_first_adam_step_closed_form():
    g = [np.array([0.5, -2.0, 1e-3])]
    p, m, v = mlp.adam_step([np.zeros(3)], g, [np.zeros(3)], [np.zeros(3)], step=1, lr=0.01)
    assert np.allclose(p[0], -0.01 * g[0] / (np.abs(g[0]) + 1e-8))
