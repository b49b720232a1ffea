"""Band features of a pair from their definition: TEST INFRASTRUCTURE ONLY.

The learned band (not in the paper; an exactness-preserving extension of its
global alignment) reads a 64-bin histogram of where shared k-mers fall
relative to the straight line from (0, 0) to (n, m):

* k = 12 letters of a DNA sequence (codes 0..3) form a 24-bit key, first
  letter in the lowest bits;
* the query contributes the k-mers starting at positions i = 0, t, 2t, ...
  with stride t = 4 * ceil(n / 16384) (at most 4,097 sampled k-mers); a key
  seen at several such positions keeps the smallest one;
* every subject k-mer start j whose key occurs in the query gives a hit
  (i, j) with the integer deviation D = (j - i) * n - (m - n) * i (that is n
  times the offset from the straight line);
* magnitude bucket of |D| / n (integer division): 0 for 0, otherwise
  1 + 2 * floor(log2(x)) + (second highest bit of x), capped at 31; bin
  32 + bucket for D >= 0 and 31 - bucket for D < 0;
* counts divided by the number of sampled query k-mers in float32 (all zero
  when a sequence is shorter than k), so the total mass measures similarity.

All binning is integer arithmetic, so any correct implementation produces the
same bins; the one float operation is a correctly rounded float32 division.
"""
from __future__ import annotations

import numpy as np

K = 12
STRIDE = 4
NBINS = 64


def stride(n: int) -> int:
    return STRIDE * max(1, -(-n // 16384))


def bucket(x: int) -> int:
    if x == 0:
        return 0
    lg = x.bit_length() - 1
    second = (x >> (lg - 1)) & 1 if lg >= 1 else 0
    return min(31, 1 + 2 * lg + second)


def kmer_keys(codes: np.ndarray) -> np.ndarray:
    """Key of the k-mer starting at every position (len - K + 1 values)."""
    c = np.asarray(codes, dtype=np.int64)
    if len(c) < K:
        return np.zeros(0, dtype=np.int64)
    keys = np.zeros(len(c) - K + 1, dtype=np.int64)
    for t in range(K):
        keys |= c[t:len(c) - K + 1 + t] << (2 * t)
    return keys


def histogram_counts(q, s) -> np.ndarray:
    """Integer hit counts per bin (int64, 64 values)."""
    n, m = len(q), len(s)
    counts = np.zeros(NBINS, dtype=np.int64)
    if n < K or m < K:
        return counts
    qk = kmer_keys(q)
    first: dict[int, int] = {}
    for i in range(0, len(qk), stride(n)):
        first.setdefault(int(qk[i]), i)
    for j, key in enumerate(kmer_keys(s)):
        i = first.get(int(key))
        if i is None:
            continue
        d = (j - i) * n - (m - n) * i
        b = bucket(abs(d) // n)
        counts[32 + b if d >= 0 else 31 - b] += 1
    return counts


def sampled(n: int) -> int:
    """Number of sampled query k-mers."""
    return 0 if n < K else (n - K) // stride(n) + 1


def features(q, s) -> np.ndarray:
    counts = histogram_counts(q, s)
    nk = sampled(len(q)) if len(s) >= K else 0
    if nk == 0:
        return np.zeros(NBINS, dtype=np.float32)
    return (counts.astype(np.float32) / np.float32(nk)).astype(np.float32)


def features_batch(batch) -> np.ndarray:
    return np.stack([features(*batch.pair(p)) for p in range(batch.n_pairs)]) if batch.n_pairs else \
        np.zeros((0, NBINS), np.float32)
