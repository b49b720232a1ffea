"""Seeded synthetic inputs for the alignment workloads.

This module only draws random sequences; it computes nothing of the alignment
method. Both the CPU oracle and the CUDA path take their inputs from here, so a
parity test compares the two on byte-identical data.

Randomness is counter-based so that a value depends only on (seed, stream,
index), never on call order or platform: SplitMix64 (Steele, Lea, Flood 2014,
"Fast splittable pseudorandom number generators") applied to
``seed_key(seed, stream) + index``. It is written with numpy uint64 arithmetic,
which wraps modulo 2**64 exactly like the published C definition.

Workloads (shapes of the paper's use cases, Sec. V: long genome pairs and
150-bp Illumina-style reads; the datasets themselves are not available, these
stand in for them):

* ``single_pair``     1,000 x 1,100 uniform ACGT (seed 0)
* ``short_reads``     262,144 read/target pairs, query 100..250 bp, target =
                      query with 4 % substitutions, 1 % indel events
                      (Geometric(0.5) lengths) and 20-bp random flanks
* ``protein_pairs``   65,536 pairs over 20 letters, log-uniform 50..1000,
                      30 % substitutions, 3 % indels, plus a seeded symmetric
                      20 x 20 int8 substitution matrix
* ``long_pair``       1 Mbp reference and a copy with 1 % substitutions,
                      0.1 % indels (Geometric(0.3)) and two 10-kbp inversions
* ``band_pairs``      65,536 pairs log-uniform 1..10 kbp with per-pair
                      substitution rate U[0,0.15], indel rate U[0,0.10]
                      (Geometric(0.3)); 5 % unrelated pairs
* ``serving_mix``     Poisson arrivals of pairs: 70 % 100-300 bp, 25 % 1-10 kbp,
                      5 % 50-200 kbp
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)

DNA = "ACGT"
COMPLEMENT = np.array([3, 2, 1, 0], dtype=np.uint8)  # A<->T, C<->G on codes 0..3


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        return z ^ (z >> np.uint64(31))


def seed_key(seed: int, stream: int) -> np.uint64:
    """Key of one random stream: SplitMix64 of (seed, stream)."""
    z = np.array([(int(seed) * 0x100000001B3 + int(stream) * 0x9E3779B97F4A7C15)
                  & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return _mix(z)[0]


class Stream:
    """Counter-based uniform random numbers: value k = SplitMix64(key + (k+1)*golden)."""

    def __init__(self, seed: int, stream: int):
        self.key = seed_key(seed, stream)
        self.pos = 0

    def u64(self, count: int) -> np.ndarray:
        idx = np.arange(self.pos + 1, self.pos + 1 + count, dtype=np.uint64)
        self.pos += count
        with np.errstate(over="ignore"):
            return _mix(self.key + idx * _GOLDEN)

    def at(self, idx: np.ndarray) -> np.ndarray:
        """Values at explicit counter positions (does not advance the stream)."""
        with np.errstate(over="ignore"):
            return _mix(self.key + (np.asarray(idx, dtype=np.uint64) + np.uint64(1)) * _GOLDEN)

    def uniform(self, count: int) -> np.ndarray:
        """Floats in [0, 1) with 53 random bits."""
        return (self.u64(count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def integers(self, lo: int, hi: int, count: int) -> np.ndarray:
        """Integers uniform in [lo, hi] (inclusive), by multiply-shift on 32 bits."""
        span = np.uint64(hi - lo + 1)
        r = (self.u64(count) >> np.uint64(32)) * span >> np.uint64(32)
        return r.astype(np.int64) + lo

    def geometric(self, p: float | np.ndarray, count: int) -> np.ndarray:
        """Lengths >= 1 with P(L = k) = (1-p)^(k-1) p (inversion method)."""
        u = 1.0 - self.uniform(count)  # (0, 1]
        return 1 + np.floor(np.log(u) / np.log1p(-np.asarray(p, dtype=np.float64))).astype(np.int64)


@dataclass
class Batch:
    """A batch of pairs: codes concatenated, offsets of length n_pairs + 1."""
    q: np.ndarray      # uint8 codes
    q_off: np.ndarray  # int64
    s: np.ndarray
    s_off: np.ndarray
    alphabet: int = 4

    @property
    def n_pairs(self) -> int:
        return len(self.q_off) - 1

    def q_len(self) -> np.ndarray:
        return np.diff(self.q_off)

    def s_len(self) -> np.ndarray:
        return np.diff(self.s_off)

    def pair(self, p: int) -> tuple[np.ndarray, np.ndarray]:
        return (self.q[self.q_off[p]:self.q_off[p + 1]], self.s[self.s_off[p]:self.s_off[p + 1]])

    def cells(self) -> int:
        return int(np.sum(self.q_len().astype(np.int64) * self.s_len().astype(np.int64)))

    def subset(self, idx) -> "Batch":
        idx = np.asarray(idx, dtype=np.int64)
        return from_pairs([self.pair(int(p)) for p in idx], self.alphabet)


def from_pairs(pairs, alphabet: int = 4) -> Batch:
    ql = [np.asarray(a, dtype=np.uint8) for a, _ in pairs]
    sl = [np.asarray(b, dtype=np.uint8) for _, b in pairs]
    q_off = np.zeros(len(pairs) + 1, dtype=np.int64)
    s_off = np.zeros(len(pairs) + 1, dtype=np.int64)
    q_off[1:] = np.cumsum([len(a) for a in ql])
    s_off[1:] = np.cumsum([len(b) for b in sl])
    q = np.concatenate(ql) if ql and q_off[-1] else np.zeros(0, dtype=np.uint8)
    s = np.concatenate(sl) if sl and s_off[-1] else np.zeros(0, dtype=np.uint8)
    return Batch(q.astype(np.uint8), q_off, s.astype(np.uint8), s_off, alphabet)


def encode_dna(text: str) -> np.ndarray:
    table = np.full(256, 255, dtype=np.uint8)
    for k, ch in enumerate(DNA):
        table[ord(ch)] = k
        table[ord(ch.lower())] = k
    codes = table[np.frombuffer(text.encode("ascii"), dtype=np.uint8)]
    if np.any(codes == 255):
        raise ValueError("not an ACGT string")
    return codes


def decode_dna(codes) -> str:
    return "".join(DNA[int(c)] for c in codes)


def _offsets(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    off[1:] = np.cumsum(lengths)
    return off


def random_codes(st: Stream, count: int, alphabet: int) -> np.ndarray:
    """Uniform letters: four 16-bit chunks per 64-bit draw, letter = chunk*alphabet >> 16."""
    words = st.u64((count + 3) // 4)
    chunks = words.view(np.uint16)[:count].astype(np.uint32)
    return ((chunks * np.uint32(alphabet)) >> np.uint32(16)).astype(np.uint8)


def log_uniform_lengths(st: Stream, lo: int, hi: int, count: int) -> np.ndarray:
    u = st.uniform(count)
    return np.rint(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)


def mutate(codes: np.ndarray, off: np.ndarray, p_sub, p_indel, geom_p: float,
           alphabet: int, st: Stream) -> tuple[np.ndarray, np.ndarray]:
    """Copy every sequence with substitutions and indel events.

    Walking each source sequence base by base: with probability ``p_sub`` the
    base is replaced by one of the other ``alphabet - 1`` letters (uniform);
    independently, with probability ``p_indel`` an indel event starts at the
    base: half of them insert Geometric(``geom_p``) uniform random letters
    after it, the other half delete that many bases starting at it (clipped at
    the sequence end). ``p_sub``/``p_indel`` are scalars or per-sequence arrays.
    One 64-bit draw per base decides both coins (32 bits each); the rare
    follow-up draws are addressed by base index in their own streams.
    """
    total = len(codes)
    nseq = len(off) - 1
    lens = np.diff(off)
    base = st.u64(total)
    u_sub = (base >> np.uint64(32)).astype(np.float64) * (1.0 / 4294967296.0)
    u_ev = (base & np.uint64(0xFFFFFFFF)).astype(np.float64) * (1.0 / 4294967296.0)
    del base
    if np.ndim(p_sub) == 0 and np.ndim(p_indel) == 0:
        sub = u_sub < float(p_sub)
        event = u_ev < float(p_indel)
    else:
        seq_of = np.repeat(np.arange(nseq, dtype=np.int64), lens)
        sub = u_sub < np.broadcast_to(np.asarray(p_sub, dtype=np.float64), (nseq,))[seq_of]
        event = u_ev < np.broadcast_to(np.asarray(p_indel, dtype=np.float64), (nseq,))[seq_of]
        del seq_of
    del u_sub, u_ev
    key2 = Stream(int(st.key) & 0x7FFFFFFFFFFFFFFF, 101)
    key3 = Stream(int(st.key) & 0x7FFFFFFFFFFFFFFF, 102)
    out_codes = codes.copy()
    sub_pos = np.nonzero(sub)[0]
    shift = 1 + ((key2.at(sub_pos) >> np.uint64(32)) * np.uint64(alphabet - 1) >> np.uint64(32)).astype(np.int64)
    out_codes[sub_pos] = ((codes[sub_pos].astype(np.int64) + shift) % alphabet).astype(np.uint8)
    ev_pos = np.nonzero(event)[0]
    r = key3.at(ev_pos)
    is_ins = (r >> np.uint64(63)) == np.uint64(0)
    u_len = 1.0 - ((r & np.uint64(0xFFFFFFFFFFFF)).astype(np.float64) + 0.5) / 281474976710656.0
    ev_len = 1 + np.floor(np.log1p(-u_len) / np.log1p(-geom_p)).astype(np.int64)
    ins_pos, ins_len = ev_pos[is_ins], ev_len[is_ins]
    dstart, dlen = ev_pos[~is_ins], ev_len[~is_ins]
    # deletions: mark [k, min(k+L, end of its sequence)) as removed
    seq_end = off[1:][np.searchsorted(off, dstart, side="right") - 1]
    dstop = np.minimum(dstart + dlen, seq_end)
    diff = (np.bincount(dstart, minlength=total + 1)
            - np.bincount(dstop, minlength=total + 1))
    keep = np.cumsum(diff[:-1]) <= 0
    slots = keep.astype(np.int64)
    slots[ins_pos] += ins_len
    csum = np.concatenate([[0], np.cumsum(slots)])
    start = csum[:-1]
    out_total = int(csum[-1])
    out = np.empty(out_total, dtype=np.uint8)
    is_orig = np.zeros(out_total, dtype=bool)
    kpos = start[keep]
    out[kpos] = out_codes[keep]
    is_orig[kpos] = True
    fill = np.nonzero(~is_orig)[0]
    out[fill] = random_codes_at(st, fill, alphabet)
    return out, csum[off].astype(np.int64)


def random_codes_at(st: Stream, idx: np.ndarray, alphabet: int) -> np.ndarray:
    """Uniform letters at explicit positions of a fresh sub-stream of ``st``."""
    sub = Stream(int(st.key) & 0x7FFFFFFFFFFFFFFF, 103)
    r = (sub.at(idx) >> np.uint64(32)) * np.uint64(alphabet) >> np.uint64(32)
    return r.astype(np.uint8)


def add_flanks(codes: np.ndarray, off: np.ndarray, flank: int, alphabet: int,
               st: Stream) -> tuple[np.ndarray, np.ndarray]:
    """Surround every sequence with ``flank`` uniform random letters on each side."""
    lens = np.diff(off)
    new_lens = lens + 2 * flank
    new_off = _offsets(new_lens)
    out = random_codes(st, int(new_off[-1]), alphabet)
    nseq = len(lens)
    seq_of = np.repeat(np.arange(nseq, dtype=np.int64), lens)
    local = np.arange(len(codes), dtype=np.int64) - off[:-1][seq_of]
    out[new_off[:-1][seq_of] + flank + local] = codes
    return out, new_off


# --------------------------------------------------------------------------- workloads

def single_pair(seed: int = 0, n: int = 1000, m: int = 1100) -> Batch:
    st = Stream(seed, 1)
    q = random_codes(st, n, 4)
    s = random_codes(st, m, 4)
    return Batch(q, np.array([0, n], dtype=np.int64), s, np.array([0, m], dtype=np.int64), 4)


def short_reads(n_pairs: int = 262144, seed: int = 2, len_lo: int = 100, len_hi: int = 250,
                p_sub: float = 0.04, p_indel: float = 0.01, flank: int = 20) -> Batch:
    st = Stream(seed, 2)
    lens = st.integers(len_lo, len_hi, n_pairs)
    q_off = _offsets(lens)
    q = random_codes(st, int(q_off[-1]), 4)
    t, t_off = mutate(q, q_off, p_sub, p_indel, 0.5, 4, st)
    s, s_off = add_flanks(t, t_off, flank, 4, st)
    return Batch(q, q_off, s, s_off, 4)


def protein_matrix(seed: int = 3, alphabet: int = 20) -> np.ndarray:
    """Symmetric int8 matrix: diagonal uniform [4, 11], off-diagonal uniform [-4, 3]."""
    st = Stream(seed, 7)
    mat = np.zeros((alphabet, alphabet), dtype=np.int8)
    diag = st.integers(4, 11, alphabet)
    off = st.integers(-4, 3, alphabet * alphabet)
    k = 0
    for a in range(alphabet):
        mat[a, a] = diag[a]
        for b in range(a + 1, alphabet):
            mat[a, b] = mat[b, a] = off[k]
            k += 1
    return mat


def protein_pairs(n_pairs: int = 65536, seed: int = 3, len_lo: int = 50, len_hi: int = 1000,
                  p_sub: float = 0.30, p_indel: float = 0.03) -> Batch:
    st = Stream(seed, 3)
    lens = log_uniform_lengths(st, len_lo, len_hi, n_pairs)
    q_off = _offsets(lens)
    q = random_codes(st, int(q_off[-1]), 20)
    s, s_off = mutate(q, q_off, p_sub, p_indel, 0.5, 20, st)
    return Batch(q, q_off, s, s_off, 20)


def long_pair(seed: int = 4, n: int = 1_000_000, p_sub: float = 0.01, p_indel: float = 0.001,
              inversion: int = 10_000, n_inversions: int = 2) -> Batch:
    st = Stream(seed, 4)
    r = random_codes(st, n, 4)
    s, s_off = mutate(r, np.array([0, n], dtype=np.int64), p_sub, p_indel, 0.3, 4, st)
    s = s.copy()
    m = len(s)
    if n_inversions and m >= n_inversions * inversion * 2:
        # non-overlapping segments: one start drawn in each of n_inversions equal slices
        slice_len = m // n_inversions
        starts = st.integers(0, slice_len - inversion, n_inversions) + np.arange(n_inversions) * slice_len
        for a in starts:
            seg = s[a:a + inversion]
            s[a:a + inversion] = COMPLEMENT[seg[::-1]]
    return Batch(r, np.array([0, n], dtype=np.int64), s, np.array([0, m], dtype=np.int64), 4)


def band_pairs(n_pairs: int = 65536, seed: int = 5, len_lo: int = 1000, len_hi: int = 10000,
               max_sub: float = 0.15, max_indel: float = 0.10, unrelated: float = 0.05) -> Batch:
    st = Stream(seed, 5)
    lens = log_uniform_lengths(st, len_lo, len_hi, n_pairs)
    q_off = _offsets(lens)
    q = random_codes(st, int(q_off[-1]), 4)
    p_sub = st.uniform(n_pairs) * max_sub
    p_indel = st.uniform(n_pairs) * max_indel
    t, t_off = mutate(q, q_off, p_sub, p_indel, 0.3, 4, st)
    is_unrel = st.uniform(n_pairs) < unrelated
    if np.any(is_unrel):
        ulen = log_uniform_lengths(st, len_lo, len_hi, n_pairs)
        tl = np.diff(t_off)
        new_len = np.where(is_unrel, ulen, tl)
        new_off = _offsets(new_len)
        out = random_codes(st, int(new_off[-1]), 4)
        seq_of = np.repeat(np.arange(n_pairs, dtype=np.int64), tl)
        sel = ~is_unrel[seq_of]
        local = np.arange(len(t), dtype=np.int64) - t_off[:-1][seq_of]
        out[new_off[:-1][seq_of[sel]] + local[sel]] = t[sel]
        t, t_off = out, new_off
    return Batch(q, q_off, t, t_off, 4)


@dataclass
class Arrivals:
    times: np.ndarray  # seconds, increasing
    batch: Batch
    kind: np.ndarray   # 0 short, 1 medium, 2 long


def serving_mix(n_requests: int, rate_per_s: float, seed: int = 6) -> Arrivals:
    """Poisson arrivals: 70 % 100-300 bp, 25 % 1-10 kbp, 5 % 50-200 kbp related pairs."""
    st = Stream(seed, 6)
    gaps = -np.log(1.0 - st.uniform(n_requests)) / rate_per_s
    times = np.cumsum(gaps)
    u = st.uniform(n_requests)
    kind = np.where(u < 0.70, 0, np.where(u < 0.95, 1, 2)).astype(np.int64)
    lo = np.array([100, 1000, 50000])[kind]
    hi = np.array([300, 10000, 200000])[kind]
    uu = st.uniform(n_requests)
    lens = np.rint(np.exp(np.log(lo) + uu * (np.log(hi) - np.log(lo)))).astype(np.int64)
    q_off = _offsets(lens)
    q = random_codes(st, int(q_off[-1]), 4)
    s, s_off = mutate(q, q_off, 0.05, 0.01, 0.3, 4, st)
    return Arrivals(times, Batch(q, q_off, s, s_off, 4), kind)


def random_pairs(n_pairs: int, len_lo: int, len_hi: int, alphabet: int = 4, seed: int = 11,
                 related: float = 0.5, p_sub: float = 0.1, p_indel: float = 0.05) -> Batch:
    """Test pairs: lengths uniform in [len_lo, len_hi]; a fraction are mutated copies."""
    st = Stream(seed, 9)
    lens = st.integers(len_lo, len_hi, n_pairs)
    q_off = _offsets(lens)
    q = random_codes(st, int(q_off[-1]), alphabet)
    t, t_off = mutate(q, q_off, p_sub, p_indel, 0.5, alphabet, st)
    slens = st.integers(len_lo, len_hi, n_pairs)
    r_off = _offsets(slens)
    r = random_codes(st, int(r_off[-1]), alphabet)
    rel = st.uniform(n_pairs) < related
    pairs = []
    for p in range(n_pairs):
        a = q[q_off[p]:q_off[p + 1]]
        b = t[t_off[p]:t_off[p + 1]] if rel[p] else r[r_off[p]:r_off[p + 1]]
        pairs.append((a, b))
    return from_pairs(pairs, alphabet)
