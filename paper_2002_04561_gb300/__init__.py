"""GB300 (sm_103a) pairwise DP alignment: Python binding of the C ABI.

The binding only marshals arguments: it passes pointers of torch tensors (or
numpy arrays for host buffers) and the current CUDA stream to the functions
declared in include/anyseq.h, with the same names. Every step of the
alignment runs in the CUDA library ``_lib/libanyseq.so``; there is no CPU
fallback, and importing the binding fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

GLOBAL, LOCAL, SEMIGLOBAL = 0, 1, 2
MODES = {"global": GLOBAL, "local": LOCAL, "semiglobal": SEMIGLOBAL}
WANT_SCORE, WANT_END, WANT_CIGAR, BAND_LEARNED = 1, 2, 4, 8
FLAG_INT32, FLAG_BAND_ACCEPTED, FLAG_FULL_FALLBACK = 1, 2, 4
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_ALPHABET", 3: "ERR_BUDGET", 4: "ERR_CUDA",
          5: "ERR_TIMEOUT", 6: "ERR_CAPACITY"}

LIB_PATH = _build.LIB


class AnyseqError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Scoring(ctypes.Structure):
    """anyseq_scoring_t. ``matrix`` (optional) must stay alive during calls."""
    _fields_ = [("alphabet", ctypes.c_int32), ("matrix", ctypes.c_void_p),
                ("match", ctypes.c_int32), ("mismatch", ctypes.c_int32),
                ("gap_open", ctypes.c_int32), ("gap_extend", ctypes.c_int32)]

    @classmethod
    def make(cls, match=2, mismatch=-1, gap_open=0, gap_extend=-1, matrix=None, alphabet=4):
        sc = cls()
        sc.alphabet = alphabet
        sc.match, sc.mismatch, sc.gap_open, sc.gap_extend = match, mismatch, gap_open, gap_extend
        if matrix is not None:
            sc._mat = np.ascontiguousarray(matrix, dtype=np.int8)
            sc.matrix = sc._mat.ctypes.data
            sc.alphabet = sc._mat.shape[0]
        else:
            sc.matrix = None
        return sc


class Result(ctypes.Structure):
    _fields_ = [("score", ctypes.c_int32), ("beg_q", ctypes.c_int32), ("beg_s", ctypes.c_int32),
                ("end_q", ctypes.c_int32), ("end_s", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("cigar_off", ctypes.c_uint64), ("cigar_len", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


RESULT_DTYPE = np.dtype([("score", np.int32), ("beg_q", np.int32), ("beg_s", np.int32),
                         ("end_q", np.int32), ("end_s", np.int32), ("flags", np.uint32),
                         ("cigar_off", np.uint64), ("cigar_len", np.uint32), ("reserved", np.uint32)])
assert RESULT_DTYPE.itemsize == ctypes.sizeof(Result) == 40

_lib = None
EXPORTS = ["anyseq_create", "anyseq_destroy", "anyseq_align_batch", "anyseq_align_long",
           "anyseq_set_option", "anyseq_get_stat", "anyseq_encode_dna", "anyseq_last_error",
           "anyseq_version", "anyseq_band_features", "anyseq_band_model_get", "anyseq_band_model_set",
           "anyseq_band_model_save", "anyseq_band_model_load", "anyseq_band_forward",
           "anyseq_band_gradient", "anyseq_band_train", "anyseq_align_long_noalloc",
           "anyseq_server_create", "anyseq_server_submit", "anyseq_server_wait", "anyseq_server_stat",
           "anyseq_server_destroy", "anyseq_plan_create", "anyseq_plan_buffers", "anyseq_plan_run",
           "anyseq_plan_wait", "anyseq_plan_destroy", "anyseq_gapped", "anyseq_autotune",
           "anyseq_autotune_table", "anyseq_autotune_set_table", "anyseq_shard_plan", "anyseq_plan_upload",
           "anyseq_plan_download"]
NOALLOC_MAX_LEN = 1048576
BAND_FEATURES = 64
BAND_PARAMS = 25090


class ServerConfig(ctypes.Structure):
    """anyseq_server_config_t."""
    _fields_ = [("device", ctypes.c_int32), ("mode", ctypes.c_int32), ("scoring", Scoring),
                ("max_batch_pairs", ctypes.c_int64), ("max_wait_us", ctypes.c_int64),
                ("long_cells", ctypes.c_int64), ("mem_budget_bytes", ctypes.c_size_t)]


def load(build_if_missing: bool = False):
    """Load libanyseq.so (optionally building it first). Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise ImportError(f"CUDA library {LIB_PATH} is missing: run paper_2002_04561_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32, U32, U64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
    lib.anyseq_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_size_t]
    lib.anyseq_destroy.argtypes = [P]
    lib.anyseq_align_batch.argtypes = [P, P, P, P, P, I64, P, I32, U32, P, P, U64, P, P]
    lib.anyseq_align_long.argtypes = [P, P, I64, P, I64, P, I32, U32, P, P, U64, P, P]
    lib.anyseq_set_option.argtypes = [P, ctypes.c_char_p, I64]
    lib.anyseq_get_stat.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double)]
    lib.anyseq_encode_dna.argtypes = [P, P, I64]
    F32 = ctypes.c_float
    lib.anyseq_band_features.argtypes = [P, P, P, P, P, I64, P, P]
    lib.anyseq_band_model_get.argtypes = [P, P, I64]
    lib.anyseq_band_model_set.argtypes = [P, P, I64]
    lib.anyseq_band_model_save.argtypes = [P, ctypes.c_char_p]
    lib.anyseq_band_model_load.argtypes = [P, ctypes.c_char_p]
    lib.anyseq_band_forward.argtypes = [P, P, I64, P, P]
    lib.anyseq_band_gradient.argtypes = [P, P, P, I64, P, P, P]
    lib.anyseq_band_train.argtypes = [P, P, P, P, P, I64, P, I32, F32, P, P]
    lib.anyseq_align_long_noalloc.argtypes = [P, I64, P, I64, P, P, P]
    lib.anyseq_server_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(ServerConfig)]
    lib.anyseq_server_submit.argtypes = [P, P, I64, P, I64, ctypes.POINTER(U64)]
    lib.anyseq_server_wait.argtypes = [P, U64, I64, P, ctypes.POINTER(I64)]
    lib.anyseq_server_stat.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double)]
    lib.anyseq_server_destroy.argtypes = [P]
    lib.anyseq_plan_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, P, P, I64, P, I32]
    lib.anyseq_plan_buffers.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P)]
    lib.anyseq_plan_run.argtypes = [P, P]
    lib.anyseq_plan_upload.argtypes = [P, P, P, P]
    lib.anyseq_plan_download.argtypes = [P, P, P]
    lib.anyseq_plan_wait.argtypes = [P, P]
    lib.anyseq_plan_destroy.argtypes = [P]
    lib.anyseq_autotune.argtypes = [P, P, P, P, P, I64, P, I32, P]
    lib.anyseq_autotune_table.argtypes = [P, P]
    lib.anyseq_autotune_set_table.argtypes = [P, P]
    lib.anyseq_gapped.argtypes = [P, I64, P, I64, I32, I32, P, U32, ctypes.c_char_p, I32, P, P, I64,
                                  ctypes.POINTER(I64)]
    lib.anyseq_shard_plan.argtypes = [P, P, I64, I32, I32, P, I64, ctypes.POINTER(I64)]
    lib.anyseq_last_error.restype = ctypes.c_char_p
    lib.anyseq_last_error.argtypes = []
    lib.anyseq_version.restype = ctypes.c_char_p
    for name in ["anyseq_create", "anyseq_destroy", "anyseq_align_batch", "anyseq_align_long",
                 "anyseq_set_option", "anyseq_get_stat", "anyseq_encode_dna", "anyseq_band_features",
                 "anyseq_band_model_get", "anyseq_band_model_set", "anyseq_band_model_save",
                 "anyseq_band_model_load", "anyseq_band_forward", "anyseq_band_gradient", "anyseq_band_train",
                 "anyseq_align_long_noalloc", "anyseq_server_create", "anyseq_server_submit",
                 "anyseq_server_wait", "anyseq_server_stat", "anyseq_server_destroy", "anyseq_plan_create",
                 "anyseq_plan_buffers", "anyseq_plan_run", "anyseq_plan_wait", "anyseq_plan_destroy",
                 "anyseq_gapped", "anyseq_autotune", "anyseq_autotune_table",
                 "anyseq_autotune_set_table", "anyseq_shard_plan", "anyseq_plan_upload", "anyseq_plan_download"]:
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise AnyseqError(status, load().anyseq_last_error().decode())


def _ptr(x) -> int | None:
    """Address of a torch tensor or numpy array (None for empty/None)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr() if x.numel() else None
    return x.ctypes.data if x.size else None


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


class Context:
    """anyseq_ctx: device, scratch arena and memory budget."""

    def __init__(self, device: int = 0, mem_budget: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.anyseq_create(ctypes.byref(h), device, mem_budget))
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            load().anyseq_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key: str, value: int):
        _check(load().anyseq_set_option(self.h, key.encode(), int(value)))

    def stat(self, key: str) -> float:
        v = ctypes.c_double(0)
        _check(load().anyseq_get_stat(self.h, key.encode(), ctypes.byref(v)))
        return v.value

    def align_batch(self, q, q_off, s, s_off, scoring: Scoring, mode: int = GLOBAL,
                    want: int = WANT_SCORE | WANT_END, out=None, cigar=None, stream=None):
        """anyseq_align_batch. Arrays: torch tensors (device or host) or numpy (host).

        Returns (out, cigar_used). ``out`` defaults to a host numpy array of RESULT_DTYPE.
        """
        n_pairs = len(q_off) - 1
        if out is None:
            out = np.zeros(n_pairs, dtype=RESULT_DTYPE)
        used = ctypes.c_uint64(0)
        cap = 0 if cigar is None else (cigar.numel() if hasattr(cigar, "numel") else cigar.size)
        _check(load().anyseq_align_batch(
            self.h, _ptr(q), _ptr(q_off), _ptr(s), _ptr(s_off), n_pairs, ctypes.byref(scoring), mode, want,
            _ptr(out), _ptr(cigar), cap, ctypes.byref(used), _stream_handle(stream)))
        return out, used.value

    def align_long(self, q, s, scoring: Scoring, mode: int = GLOBAL, want: int = WANT_SCORE | WANT_END,
                   out=None, cigar=None, stream=None):
        """anyseq_align_long on one pair. Returns (out, cigar_used)."""
        n = q.numel() if hasattr(q, "numel") else len(q)
        m = s.numel() if hasattr(s, "numel") else len(s)
        if out is None:
            out = np.zeros(1, dtype=RESULT_DTYPE)
        used = ctypes.c_uint64(0)
        cap = 0 if cigar is None else (cigar.numel() if hasattr(cigar, "numel") else cigar.size)
        _check(load().anyseq_align_long(
            self.h, _ptr(q), n, _ptr(s), m, ctypes.byref(scoring), mode, want, _ptr(out), _ptr(cigar), cap,
            ctypes.byref(used), _stream_handle(stream)))
        return out, used.value


    # ---------------------------------------------------------------- autotuner
    def autotune(self, q, q_off, s, s_off, scoring: Scoring, mode: int = GLOBAL, stream=None):
        """anyseq_autotune on a sample; returns the 256 per-bin caps (0 = default)."""
        _check(load().anyseq_autotune(self.h, _ptr(q), _ptr(q_off), _ptr(s), _ptr(s_off), len(q_off) - 1,
                                      ctypes.byref(scoring), mode, _stream_handle(stream)))
        caps = np.zeros(256, dtype=np.uint8)
        _check(load().anyseq_autotune_table(self.h, _ptr(caps)))
        return caps

    def autotune_set_table(self, caps):
        """anyseq_autotune_set_table: install a saved table of 256 caps."""
        caps = np.ascontiguousarray(caps, dtype=np.uint8)
        if caps.shape != (256,):
            raise ValueError("the table holds 256 caps")
        _check(load().anyseq_autotune_set_table(self.h, _ptr(caps)))

    # ---------------------------------------------------------------- learned band
    def band_features(self, q, q_off, s, s_off, out=None, stream=None):
        n_pairs = len(q_off) - 1
        if out is None:
            out = np.zeros((n_pairs, BAND_FEATURES), dtype=np.float32)
        _check(load().anyseq_band_features(self.h, _ptr(q), _ptr(q_off), _ptr(s), _ptr(s_off), n_pairs,
                                           _ptr(out), _stream_handle(stream)))
        return out

    def band_model_get(self) -> np.ndarray:
        out = np.zeros(BAND_PARAMS, dtype=np.float32)
        _check(load().anyseq_band_model_get(self.h, _ptr(out), BAND_PARAMS))
        return out

    def band_model_set(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32)
        _check(load().anyseq_band_model_set(self.h, _ptr(params), params.size))

    def band_model_save(self, path: str):
        _check(load().anyseq_band_model_save(self.h, path.encode()))

    def band_model_load(self, path: str):
        _check(load().anyseq_band_model_load(self.h, path.encode()))

    def band_forward(self, x, stream=None) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.zeros((x.shape[0], 2), dtype=np.float32)
        _check(load().anyseq_band_forward(self.h, _ptr(x), x.shape[0], _ptr(y), _stream_handle(stream)))
        return y

    def band_gradient(self, x, targets, stream=None):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(targets, dtype=np.float32)
        g = np.zeros(BAND_PARAMS, dtype=np.float32)
        loss = ctypes.c_float(0)
        _check(load().anyseq_band_gradient(self.h, _ptr(x), _ptr(t), x.shape[0], _ptr(g), ctypes.byref(loss),
                                           _stream_handle(stream)))
        return float(loss.value), g

    def band_train(self, q, q_off, s, s_off, scoring: Scoring, epochs: int = 30, lr: float = 1e-3, stream=None):
        loss = ctypes.c_float(0)
        _check(load().anyseq_band_train(self.h, _ptr(q), _ptr(q_off), _ptr(s), _ptr(s_off), len(q_off) - 1,
                                        ctypes.byref(scoring), epochs, lr, ctypes.byref(loss),
                                        _stream_handle(stream)))
        return float(loss.value)


def align_long_noalloc(q, s, scoring: Scoring, score, stream=None):
    """anyseq_align_long_noalloc: global score of one long pair into the device
    int32 tensor ``score``, with no device allocation by the library (for
    callers whose device memory is owned by someone else; see the header)."""
    n = q.numel() if hasattr(q, "numel") else len(q)
    m = s.numel() if hasattr(s, "numel") else len(s)
    lib = load()
    dev = getattr(q, "device", None)
    if dev is not None and dev.type == "cuda":
        # the library uses the current device's scratch array: make q's device current
        import torch
        with torch.cuda.device(dev):
            _check(lib.anyseq_align_long_noalloc(_ptr(q), n, _ptr(s), m, ctypes.byref(scoring), _ptr(score),
                                                 _stream_handle(stream)))
        return
    _check(lib.anyseq_align_long_noalloc(_ptr(q), n, _ptr(s), m, ctypes.byref(scoring), _ptr(score),
                                         _stream_handle(stream)))


def gapped(q, s, beg_q: int, beg_s: int, cigar, letters: str = "ACGT"):
    """anyseq_gapped: the two aligned strings ('-' against gaps) of one result."""
    q = np.ascontiguousarray(q, dtype=np.uint8)
    s = np.ascontiguousarray(s, dtype=np.uint8)
    cigar = np.ascontiguousarray(cigar, dtype=np.uint32)
    n = ctypes.c_int64(0)
    cap = q.size + s.size + 1
    qo, so = ctypes.create_string_buffer(cap), ctypes.create_string_buffer(cap)
    _check(load().anyseq_gapped(_ptr(q), q.size, _ptr(s), s.size, beg_q, beg_s, _ptr(cigar), cigar.size,
                                letters.encode(), len(letters), qo, so, cap, ctypes.byref(n)))
    return qo.value.decode(), so.value.decode()


def shard_plan(q_off, s_off, world: int, rank: int) -> np.ndarray:
    """anyseq_shard_plan: the pair indices (int64, increasing) that rank
    ``rank`` of ``world`` aligns from a batch with these host offsets."""
    q_off = np.ascontiguousarray(q_off, dtype=np.int64)
    s_off = np.ascontiguousarray(s_off, dtype=np.int64)
    n = len(q_off) - 1
    cap = max(1, -(-n // max(1, world)))
    idx = np.zeros(cap, dtype=np.int64)
    count = ctypes.c_int64(0)
    _check(load().anyseq_shard_plan(_ptr(q_off), _ptr(s_off), n, world, rank, _ptr(idx), cap, ctypes.byref(count)))
    return idx[:count.value].copy()


def encode_dna(text: str) -> np.ndarray:
    raw = text.encode("ascii")
    out = np.zeros(len(raw), dtype=np.uint8)
    _check(load().anyseq_encode_dna(raw, _ptr(out), len(raw)))
    return out


def version() -> str:
    return load().anyseq_version().decode()


class Server:
    """anyseq_server: a request queue drained in micro-batches by a native worker
    thread (score and optimum cell per pair). ``submit`` and ``wait`` may be
    called from any thread; both release the GIL while in the library."""

    def __init__(self, scoring: Scoring, mode: int = GLOBAL, device: int = 0, max_batch_pairs: int = 0,
                 max_wait_us: int = 0, long_cells: int = 0, mem_budget: int = 0):
        lib = load()
        self._cfg = ServerConfig(device, mode, scoring, max_batch_pairs, max_wait_us, long_cells, mem_budget)
        self._scoring = scoring  # keeps a matrix alive until the server has copied it
        h = ctypes.c_void_p()
        _check(lib.anyseq_server_create(ctypes.byref(h), ctypes.byref(self._cfg)))
        self.h = h

    def submit(self, q, s) -> int:
        q = np.ascontiguousarray(q, dtype=np.uint8)
        s = np.ascontiguousarray(s, dtype=np.uint8)
        t = ctypes.c_uint64(0)
        _check(load().anyseq_server_submit(self.h, _ptr(q), q.size, _ptr(s), s.size, ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_us: int = -1):
        """Returns (result record, latency in ns)."""
        out = np.zeros(1, dtype=RESULT_DTYPE)
        lat = ctypes.c_int64(0)
        _check(load().anyseq_server_wait(self.h, ticket, timeout_us, _ptr(out), ctypes.byref(lat)))
        return out[0], lat.value

    def stat(self, key: str) -> float:
        v = ctypes.c_double(0)
        _check(load().anyseq_server_stat(self.h, key.encode(), ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "h", None):
            load().anyseq_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """anyseq_plan: one batch shape of align_batch captured in a CUDA graph.

    ``q``, ``s`` and ``out`` are torch uint8 views of the plan's device buffers
    (letters in, 40-byte result records out); ``run`` replays the graph on the
    current stream, ``wait`` synchronises and checks the letters."""

    def __init__(self, q_off, s_off, scoring: Scoring, mode: int = GLOBAL, device: int = 0):
        import torch
        lib = load()
        q_off = np.ascontiguousarray(q_off, dtype=np.int64)
        s_off = np.ascontiguousarray(s_off, dtype=np.int64)
        self._scoring = scoring
        h = ctypes.c_void_p()
        _check(lib.anyseq_plan_create(ctypes.byref(h), device, _ptr(q_off), _ptr(s_off), len(q_off) - 1,
                                      ctypes.byref(scoring), mode))
        self.h = h
        self.n_pairs = len(q_off) - 1
        pq, ps, po = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib.anyseq_plan_buffers(h, ctypes.byref(pq), ctypes.byref(ps), ctypes.byref(po)))
        dev = torch.device("cuda", device)

        def view(ptr, nbytes):
            # a torch view of plan-owned device memory (no copy, no ownership)
            class _Arr:
                __cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr or 0, False),
                                            "version": 3, "strides": None}
            return torch.as_tensor(_Arr(), device=dev)

        self.q = view(pq.value, int(q_off[-1]))
        self.s = view(ps.value, int(s_off[-1]))
        self.out = view(po.value, self.n_pairs * RESULT_DTYPE.itemsize)

    def run(self, stream=None):
        _check(load().anyseq_plan_run(self.h, _stream_handle(stream)))

    def upload(self, q, s, stream=None):
        """anyseq_plan_upload: the letters of the next run from q and s (torch
        tensors or numpy arrays, host or device), asynchronously on the stream."""
        _check(load().anyseq_plan_upload(self.h, _ptr(q), _ptr(s), _stream_handle(stream)))

    def download(self, out, stream=None):
        """anyseq_plan_download: the last run's result records into out (n_pairs x 40
        bytes, host or device), asynchronously on the stream; valid after wait()."""
        _check(load().anyseq_plan_download(self.h, _ptr(out), _stream_handle(stream)))

    def wait(self, stream=None):
        _check(load().anyseq_plan_wait(self.h, _stream_handle(stream)))

    def results(self):
        return self.out.cpu().numpy().view(RESULT_DTYPE)

    def close(self):
        if getattr(self, "h", None):
            load().anyseq_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
