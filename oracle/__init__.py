"""CPU oracle for pairwise DP alignment: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package. The product path (the CUDA library and its
binding) never imports it and fails loudly when its own extension is missing.

The arithmetic lives in ``anyseq_oracle.c`` (plain scalar C, int64, full
matrices for tracebacks); this file compiles it with gcc and calls it through
ctypes. Batches are split over host threads (ctypes releases the GIL), which
changes no arithmetic. ``mlp.py`` holds the float64 reference of the band
network and ``features.py`` the k-mer diagonal histogram, both from their
definitions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

GLOBAL, LOCAL, SEMIGLOBAL = 0, 1, 2
MODES = {"global": GLOBAL, "local": LOCAL, "semiglobal": SEMIGLOBAL}
OP_M, OP_I, OP_D = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "anyseq_oracle.c")
_OUT = os.path.join(_HERE, "_lib", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _OUT)
    return _OUT


class _Scoring(ctypes.Structure):
    _fields_ = [("alphabet", ctypes.c_int32), ("matrix", ctypes.c_void_p),
                ("match", ctypes.c_int32), ("mismatch", ctypes.c_int32),
                ("gap_open", ctypes.c_int32), ("gap_extend", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("score", ctypes.c_int64), ("beg_q", ctypes.c_int64), ("beg_s", ctypes.c_int64),
                ("end_q", ctypes.c_int64), ("end_s", ctypes.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.orc_score.argtypes = [P, I64, P, I64, P, ctypes.c_int, P]
            lib.orc_align.argtypes = [P, I64, P, I64, P, ctypes.c_int, P, P, I64, P]
            lib.orc_last_row.argtypes = [P, I64, P, I64, P, I64, ctypes.c_int, P, P]
            lib.orc_hirschberg.argtypes = [P, I64, P, I64, P, I64, P, I64, P, P]
            lib.orc_start_cell.argtypes = [P, I64, P, I64, P, ctypes.c_int, P, P, P]
            lib.orc_score_batch.argtypes = [P, P, P, P, I64, I64, P, ctypes.c_int, P]
            lib.orc_align_batch.argtypes = [P, P, P, P, I64, I64, P, ctypes.c_int, P, P, P, P]
            for f in (lib.orc_score, lib.orc_align, lib.orc_last_row, lib.orc_hirschberg, lib.orc_start_cell,
                      lib.orc_score_batch, lib.orc_align_batch):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Scoring:
    """Signed scores: a gap of length k adds gap_open + k * gap_extend."""
    match: int = 2
    mismatch: int = -1
    gap_open: int = 0
    gap_extend: int = -1
    matrix: np.ndarray | None = None
    alphabet: int = 4

    def __post_init__(self):
        # a matrix fixes the alphabet (its row stride in the C arrays)
        if self.matrix is not None:
            self.alphabet = int(np.asarray(self.matrix).shape[0])

    def _c(self):
        mat = None
        if self.matrix is not None:
            mat = np.ascontiguousarray(self.matrix, dtype=np.int8)
        st = _Scoring(self.alphabet, mat.ctypes.data if mat is not None else None,
                      self.match, self.mismatch, self.gap_open, self.gap_extend)
        return st, mat  # keep the matrix alive alongside the struct

    def sigma(self, a: int, b: int) -> int:
        if self.matrix is not None:
            return int(self.matrix[a, b])
        return self.match if a == b else self.mismatch


def _ptr(a: np.ndarray):
    return a.ctypes.data if a.size else None


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def score(q, s, sc: Scoring, mode: int = GLOBAL) -> tuple[int, int, int]:
    """(score, end_q, end_s) in linear space."""
    lib = _load()
    q, s = _u8(q), _u8(s)
    st, keep = sc._c()
    r = _Result()
    _check(lib.orc_score(_ptr(q), len(q), _ptr(s), len(s), ctypes.byref(st), mode, ctypes.byref(r)), "score")
    return int(r.score), int(r.end_q), int(r.end_s)


def align(q, s, sc: Scoring, mode: int = GLOBAL):
    """(score, (beg_q, beg_s), (end_q, end_s), cigar uint32 array) from full matrices."""
    lib = _load()
    q, s = _u8(q), _u8(s)
    st, keep = sc._c()
    cap = len(q) + len(s) + 2
    cig = np.zeros(cap, dtype=np.uint32)
    n_c = ctypes.c_int64(0)
    r = _Result()
    _check(lib.orc_align(_ptr(q), len(q), _ptr(s), len(s), ctypes.byref(st), mode, ctypes.byref(r),
                         _ptr(cig), cap, ctypes.byref(n_c)), "align")
    return int(r.score), (int(r.beg_q), int(r.beg_s)), (int(r.end_q), int(r.end_s)), cig[:n_c.value].copy()


def last_row(q, s, sc: Scoring, tb: int, rev: bool = False):
    """H and E of the last row of a global pass with column-0 gap open tb."""
    lib = _load()
    q, s = _u8(q), _u8(s)
    st, keep = sc._c()
    CC = np.zeros(len(s) + 1, dtype=np.int64)
    DD = np.zeros(len(s) + 1, dtype=np.int64)
    _check(lib.orc_last_row(_ptr(q), len(q), _ptr(s), len(s), ctypes.byref(st), tb, int(rev),
                            CC.ctypes.data, DD.ctypes.data), "last_row")
    return CC, DD


BASE_CELLS = 1 << 16


def hirschberg(q, s, sc: Scoring, base_cells: int = BASE_CELLS):
    """(cigar, cells relaxed) of the global alignment by the divide-and-conquer traceback."""
    lib = _load()
    q, s = _u8(q), _u8(s)
    st, keep = sc._c()
    cap = len(q) + len(s) + 2
    cig = np.zeros(cap, dtype=np.uint32)
    n_c = ctypes.c_int64(0)
    cells = ctypes.c_int64(0)
    _check(lib.orc_hirschberg(_ptr(q), len(q), _ptr(s), len(s), ctypes.byref(st), base_cells,
                              _ptr(cig), cap, ctypes.byref(n_c), ctypes.byref(cells)), "hirschberg")
    return cig[:n_c.value].copy(), int(cells.value)


def start_cell(q, s, sc: Scoring, mode: int):
    """(G, i, j): the start of largest G(i, j) = global score of q[i:] against
    s[j:] (local: any start; semi-global: i == 0 or j == 0), ties: largest i,
    then largest j (anyseq_oracle.c, orc_start_cell)."""
    lib = _load()
    q, s = _u8(q), _u8(s)
    st, keep = sc._c()
    g, i, j = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib.orc_start_cell(_ptr(q), len(q), _ptr(s), len(s), ctypes.byref(st), mode,
                              ctypes.byref(g), ctypes.byref(i), ctypes.byref(j)), "start_cell")
    return int(g.value), int(i.value), int(j.value)


def long_alignment(q, s, sc: Scoring, mode: int = GLOBAL, base_cells: int = BASE_CELLS):
    """The linear-space alignment of one long pair, in every mode:
    (score, (beg_q, beg_s), (end_q, end_s), cigar).

    Global: the divide-and-conquer CIGAR of the whole pair. Local and
    semi-global: the optimum cell (score()), the start cell (start_cell() over
    the prefixes ending there), and the divide-and-conquer CIGAR of the two
    substrings between them; an empty optimum (score 0) begins at its end."""
    q, s = _u8(q), _u8(s)
    if mode == GLOBAL:
        S, _, _ = score(q, s, sc, GLOBAL)
        cig, _ = hirschberg(q, s, sc, base_cells)
        return S, (0, 0), (len(q), len(s)), cig
    S, ei, ej = score(q, s, sc, mode)
    if S <= 0 or ei == 0 or ej == 0:
        return S, (ei, ej), (ei, ej), np.zeros(0, dtype=np.uint32)
    G, bi, bj = start_cell(q[:ei], s[:ej], sc, mode)
    if G != S:
        raise RuntimeError(f"oracle start cell: G = {G}, optimum {S}")
    cig, _ = hirschberg(q[bi:ei], s[bj:ej], sc, base_cells)
    return S, (bi, bj), (ei, ej), cig


def _chunks(n: int, threads: int):
    k = max(1, min(threads * 8, n))
    bounds = np.linspace(0, n, k + 1).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def score_batch(batch, sc: Scoring, mode: int = GLOBAL, threads: int | None = None):
    """Arrays (score, end_q, end_s) for every pair of a synth.Batch."""
    lib = _load()
    threads = threads or default_threads()
    q, s = _u8(batch.q), _u8(batch.s)
    q_off = np.ascontiguousarray(batch.q_off, dtype=np.int64)
    s_off = np.ascontiguousarray(batch.s_off, dtype=np.int64)
    n = len(q_off) - 1
    res = (_Result * max(n, 1))()
    st, keep = sc._c()

    def run(ab):
        a, b = ab
        return lib.orc_score_batch(_ptr(q), q_off.ctypes.data, _ptr(s), s_off.ctypes.data, a, b,
                                   ctypes.byref(st), mode, ctypes.addressof(res))

    with ThreadPoolExecutor(threads) as ex:
        for rc in ex.map(run, _chunks(n, threads)):
            _check(rc, "score_batch")
    arr = np.frombuffer(res, dtype=np.int64).reshape(-1, 5)[:n]
    return arr[:, 0].copy(), arr[:, 3].copy(), arr[:, 4].copy()


def align_batch(batch, sc: Scoring, mode: int = GLOBAL, threads: int | None = None):
    """Per pair: results (score, beg_q, beg_s, end_q, end_s) and a list of CIGAR arrays."""
    lib = _load()
    threads = threads or default_threads()
    q, s = _u8(batch.q), _u8(batch.s)
    q_off = np.ascontiguousarray(batch.q_off, dtype=np.int64)
    s_off = np.ascontiguousarray(batch.s_off, dtype=np.int64)
    n = len(q_off) - 1
    caps = np.diff(q_off) + np.diff(s_off) + 2
    cig_off = np.zeros(n + 1, dtype=np.int64)
    cig_off[1:] = np.cumsum(caps)
    cig = np.zeros(max(int(cig_off[-1]), 1), dtype=np.uint32)
    cig_len = np.zeros(max(n, 1), dtype=np.int64)
    res = (_Result * max(n, 1))()
    st, keep = sc._c()

    def run(ab):
        a, b = ab
        return lib.orc_align_batch(_ptr(q), q_off.ctypes.data, _ptr(s), s_off.ctypes.data, a, b,
                                   ctypes.byref(st), mode, ctypes.addressof(res), cig.ctypes.data,
                                   cig_off.ctypes.data, cig_len.ctypes.data)

    with ThreadPoolExecutor(threads) as ex:
        for rc in ex.map(run, _chunks(n, threads)):
            _check(rc, "align_batch")
    arr = np.frombuffer(res, dtype=np.int64).reshape(-1, 5)[:n].copy()
    cigars = [cig[cig_off[p]:cig_off[p] + cig_len[p]].copy() for p in range(n)]
    return arr, cigars


def cigar_string(cig) -> str:
    return "".join(f"{int(w) >> 4}{'MID'[int(w) & 15]}" for w in cig)
