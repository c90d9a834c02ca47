"""Batched exact gap-affine WFA on one GB300 -- Python binding of libwfa_gpu.so.

The compute lives in hand-written CUDA (``csrc/``) behind the C ABI declared
in ``include/wfa_gpu.h``.  This module only marshals arguments into that ABI:
the functions ``wfa_gpu_*`` below have the C names and take raw addresses;
``Aligner`` wraps them for numpy host arrays and torch CUDA tensors.  There
is no fallback: if the library is missing, loading raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import synth  # noqa: F401  (seeded inputs; no alignment arithmetic)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwfa_gpu.so")

WFA_GPU_OK = 0
WFA_GPU_EINVAL = -1
WFA_GPU_ENOMEM = -2
WFA_GPU_ECUDA = -3
WFA_GPU_ECIGAR_CAPACITY = -4
WFA_GPU_ETIMEOUT = -5
WFA_PAIR_OK, WFA_PAIR_SCORE_LIMIT, WFA_PAIR_INVALID_CHAR = 0, 1, 2
WFA_GPU_SCORE_ONLY, WFA_GPU_DEVICE_PTRS, WFA_GPU_TIMING, WFA_GPU_PLAIN, WFA_GPU_GRAPH = 1, 2, 4, 8, 16
WFA_GPU_ARENA_ONLY = 32
WFA_GPU_MAX_SEQ_LEN = (1 << 28) - 1
WFA_GPU_SERVER_MERGE_PAIRS = 65536

# every function include/wfa_gpu.h declares
EXPORTS = (
    "wfa_gpu_create",
    "wfa_gpu_set_stream",
    "wfa_gpu_align_batch",
    "wfa_gpu_pack2bit",
    "wfa_gpu_cigar_bound",
    "wfa_gpu_last_timing",
    "wfa_gpu_strerror",
    "wfa_gpu_destroy",
    "wfa_gpu_align_short_noalloc",
    "wfa_gpu_server_create",
    "wfa_gpu_server_submit",
    "wfa_gpu_server_wait",
    "wfa_gpu_request_bytes",
    "wfa_gpu_server_destroy",
    "wfa_gpu_short_variant_name",
    "wfa_gpu_set_ends_free",
)
WFA_GPU_NOALLOC_SCRATCH_BYTES = 4 << 20
WFA_GPU_NOALLOC_MAX_PAIRS = 32768
WFA_GPU_NOALLOC_MAX_LEN = 127


class Penalties(ctypes.Structure):
    _fields_ = [("x", ctypes.c_int32), ("o", ctypes.c_int32), ("e", ctypes.c_int32)]


class Timing(ctypes.Structure):
    _fields_ = [
        ("h2d_ms", ctypes.c_float),
        ("align_ms", ctypes.c_float),
        ("general_ms", ctypes.c_float),
        ("cigar_ms", ctypes.c_float),
        ("d2h_ms", ctypes.c_float),
        ("total_ms", ctypes.c_float),
        ("kernel_launches", ctypes.c_int32),
        ("short_variant", ctypes.c_int32),
        ("deferred_pairs", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class Request(ctypes.Structure):
    _fields_ = [
        ("n_pairs", ctypes.c_int64),
        ("patterns", ctypes.c_void_p),
        ("pattern_offsets", ctypes.c_void_p),
        ("pattern_lengths", ctypes.c_void_p),
        ("texts", ctypes.c_void_p),
        ("text_offsets", ctypes.c_void_p),
        ("text_lengths", ctypes.c_void_p),
        ("pen", Penalties),
        ("max_score", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("out_scores", ctypes.c_void_p),
        ("out_status", ctypes.c_void_p),
        ("out_cigars", ctypes.c_void_p),
        ("cigar_capacity_words", ctypes.c_int64),
        ("out_cigar_offsets", ctypes.c_void_p),
    ]


class RequestStats(ctypes.Structure):
    _fields_ = [
        ("submit_s", ctypes.c_double),
        ("start_s", ctypes.c_double),
        ("end_s", ctypes.c_double),
        ("result", ctypes.c_int32),
        ("worker", ctypes.c_int32),
    ]


class WfaGpuError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__("%s%s (%d)" % (what + ": " if what else "", wfa_gpu_strerror(code), code))


_lib = None


def load(path: str = LIB_PATH):
    """Load libwfa_gpu.so (built by ``paper_2204_02085_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libwfa_gpu.so not built at %s: run `python -c 'import __graft_entry__ as g; g.build()'`"
                          % path)
    L = ctypes.CDLL(path)
    vp, i64, i32, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
    L.wfa_gpu_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t]
    L.wfa_gpu_create.restype = ctypes.c_int
    L.wfa_gpu_set_stream.argtypes = [vp, vp]
    L.wfa_gpu_set_stream.restype = ctypes.c_int
    L.wfa_gpu_align_batch.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, Penalties, i32, u32, vp, vp, vp, i64, vp]
    L.wfa_gpu_align_batch.restype = ctypes.c_int
    L.wfa_gpu_pack2bit.argtypes = [vp, i64, vp, vp, vp, u32, vp, i64, vp, vp]
    L.wfa_gpu_pack2bit.restype = ctypes.c_int
    L.wfa_gpu_cigar_bound.argtypes = [i32, i32, Penalties, i32]
    L.wfa_gpu_cigar_bound.restype = i64
    L.wfa_gpu_last_timing.argtypes = [vp, ctypes.POINTER(Timing)]
    L.wfa_gpu_last_timing.restype = ctypes.c_int
    L.wfa_gpu_strerror.argtypes = [ctypes.c_int]
    L.wfa_gpu_strerror.restype = ctypes.c_char_p
    L.wfa_gpu_destroy.argtypes = [vp]
    L.wfa_gpu_destroy.restype = None
    L.wfa_gpu_short_variant_name.argtypes = [vp, ctypes.c_int]
    L.wfa_gpu_short_variant_name.restype = ctypes.c_char_p
    L.wfa_gpu_set_ends_free.argtypes = [vp, i32, i32, i32, i32]
    L.wfa_gpu_set_ends_free.restype = ctypes.c_int
    L.wfa_gpu_align_short_noalloc.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, Penalties, i32, vp, vp, vp, i64, vp]
    L.wfa_gpu_align_short_noalloc.restype = ctypes.c_int
    L.wfa_gpu_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_size_t]
    L.wfa_gpu_server_create.restype = ctypes.c_int
    L.wfa_gpu_server_submit.argtypes = [vp, ctypes.POINTER(Request)]
    L.wfa_gpu_server_submit.restype = i64
    L.wfa_gpu_server_wait.argtypes = [vp, i64, ctypes.c_double, ctypes.POINTER(RequestStats)]
    L.wfa_gpu_server_wait.restype = ctypes.c_int
    L.wfa_gpu_request_bytes.argtypes = [ctypes.POINTER(Request)]
    L.wfa_gpu_request_bytes.restype = i64
    L.wfa_gpu_server_destroy.argtypes = [vp]
    L.wfa_gpu_server_destroy.restype = None
    _lib = L
    return L


# ----------------------------------------------------------- the C names


def wfa_gpu_create(device: int = 0, scratch_bytes: int = 0):
    """Returns (code, ctx handle or None)."""
    h = ctypes.c_void_p()
    rc = load().wfa_gpu_create(ctypes.byref(h), device, scratch_bytes)
    return rc, (h if rc == WFA_GPU_OK else None)


def wfa_gpu_set_stream(ctx, stream: int | None) -> int:
    return load().wfa_gpu_set_stream(ctx, stream or None)


def wfa_gpu_align_batch(ctx, n_pairs, patterns, pattern_offsets, pattern_lengths, texts, text_offsets,
                        text_lengths, pen, max_score, flags, out_scores, out_status, out_cigars,
                        cigar_capacity_words, out_cigar_offsets) -> int:
    """Raw call: every buffer argument is an address (int) or None."""
    if not isinstance(pen, Penalties):
        pen = Penalties(*pen)
    return load().wfa_gpu_align_batch(ctx, n_pairs, patterns, pattern_offsets, pattern_lengths, texts,
                                      text_offsets, text_lengths, pen, max_score, flags, out_scores,
                                      out_status, out_cigars, cigar_capacity_words, out_cigar_offsets)


def wfa_gpu_pack2bit(ctx, n_seqs, seqs, offsets, lengths, flags, out_words, words_capacity,
                     out_word_offsets, out_invalid) -> int:
    return load().wfa_gpu_pack2bit(ctx, n_seqs, seqs, offsets, lengths, flags, out_words, words_capacity,
                                   out_word_offsets, out_invalid)


def wfa_gpu_cigar_bound(plen: int, tlen: int, pen, max_score: int = 0) -> int:
    if not isinstance(pen, Penalties):
        pen = Penalties(*pen)
    return load().wfa_gpu_cigar_bound(plen, tlen, pen, max_score)


def wfa_gpu_short_variant_name(ctx, index: int) -> str | None:
    r = load().wfa_gpu_short_variant_name(ctx, index)
    return None if r is None else r.decode()


def wfa_gpu_last_timing(ctx) -> Timing:
    t = Timing()
    rc = load().wfa_gpu_last_timing(ctx, ctypes.byref(t))
    if rc != WFA_GPU_OK:
        raise WfaGpuError(rc, "wfa_gpu_last_timing")
    return t


def wfa_gpu_strerror(code: int) -> str:
    return load().wfa_gpu_strerror(code).decode()


def wfa_gpu_destroy(ctx) -> None:
    load().wfa_gpu_destroy(ctx)


def wfa_gpu_align_short_noalloc(stream, n_pairs, patterns, pattern_offsets, pattern_lengths, texts, text_offsets,
                                text_lengths, pen, max_score, out_scores, out_status, out_cigars,
                                cigar_capacity_words, out_cigar_offsets) -> int:
    """Raw call of the entry point that allocates nothing: device addresses
    (int) or None, ``stream`` a cudaStream_t handle (int) or None."""
    if not isinstance(pen, Penalties):
        pen = Penalties(*pen)
    return load().wfa_gpu_align_short_noalloc(stream or None, n_pairs, patterns, pattern_offsets, pattern_lengths,
                                              texts, text_offsets, text_lengths, pen, max_score, out_scores,
                                              out_status, out_cigars, cigar_capacity_words, out_cigar_offsets)


# ------------------------------------------------------------ marshalling


def _addr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    # torch tensors
    if not a.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return a.data_ptr()


class Aligner:
    """One library context.  ``align`` takes numpy host arrays (the library
    copies them to the device and back); ``align_device`` takes torch CUDA
    tensors on the context's device (no host copies)."""

    def __init__(self, device: int = 0, scratch_bytes: int = 0):
        rc, h = wfa_gpu_create(device, scratch_bytes)
        if rc != WFA_GPU_OK:
            raise WfaGpuError(rc, "wfa_gpu_create")
        self.ctx = h
        self.device = device

    def close(self):
        if self.ctx is not None:
            wfa_gpu_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream) -> None:
        """Launch on a torch.cuda.Stream (or raw cudaStream_t int); None
        restores the context's own stream."""
        handle = getattr(stream, "cuda_stream", stream)
        rc = wfa_gpu_set_stream(self.ctx, handle)
        if rc != WFA_GPU_OK:
            raise WfaGpuError(rc, "wfa_gpu_set_stream")

    def timing(self) -> dict:
        return wfa_gpu_last_timing(self.ctx).as_dict()

    def set_ends_free(self, pattern_begin: int = 0, pattern_end: int = 0, text_begin: int = 0,
                      text_end: int = 0) -> None:
        """Ends-free alignment for later calls (all 0: global)."""
        rc = load().wfa_gpu_set_ends_free(self.ctx, pattern_begin, pattern_end, text_begin, text_end)
        if rc != WFA_GPU_OK:
            raise WfaGpuError(rc, "wfa_gpu_set_ends_free")

    def variant_name(self, index: int) -> str | None:
        """Name of short-kernel variant `index` (as timing()["short_variant"])."""
        return wfa_gpu_short_variant_name(self.ctx, index)

    def align(self, batch, pen=(4, 6, 2), max_score: int = 0, score_only: bool = False,
              cigar_capacity: int | None = None, timing: bool = False, use_offsets: bool = True,
              plain: bool = False, arena_only: bool = False):
        """Host-memory call.  ``batch`` has patterns/pattern_offsets/
        pattern_lengths/texts/text_offsets/text_lengths as numpy arrays.
        Returns (scores, status, cigar words, cigar offsets)."""
        n = int(len(batch.pattern_lengths))
        pat = np.ascontiguousarray(batch.patterns, dtype=np.uint8)
        txt = np.ascontiguousarray(batch.texts, dtype=np.uint8)
        plen = np.ascontiguousarray(batch.pattern_lengths, dtype=np.int32)
        tlen = np.ascontiguousarray(batch.text_lengths, dtype=np.int32)
        poff = np.ascontiguousarray(batch.pattern_offsets, dtype=np.int64) if use_offsets else None
        toff = np.ascontiguousarray(batch.text_offsets, dtype=np.int64) if use_offsets else None
        scores = np.empty(n, dtype=np.int32)
        status = np.empty(n, dtype=np.int8)
        flags = (WFA_GPU_SCORE_ONLY if score_only else 0) | (WFA_GPU_TIMING if timing else 0) | \
            (WFA_GPU_PLAIN if plain else 0) | (WFA_GPU_ARENA_ONLY if arena_only else 0)
        offs = np.zeros(n + 1, dtype=np.int64)
        cap = 0 if score_only else int(cigar_capacity if cigar_capacity is not None else max(16 * n, 1))
        words = np.empty(max(cap, 1), dtype=np.uint32)
        while True:
            rc = wfa_gpu_align_batch(self.ctx, n, _addr(pat), _addr(poff), _addr(plen), _addr(txt), _addr(toff),
                                     _addr(tlen), pen, max_score, flags, _addr(scores), _addr(status),
                                     None if score_only else _addr(words), cap,
                                     None if score_only else _addr(offs))
            if rc == WFA_GPU_ECIGAR_CAPACITY and cigar_capacity is None:
                cap = int(offs[n])
                words = np.empty(max(cap, 1), dtype=np.uint32)
                continue
            break
        if rc != WFA_GPU_OK:
            raise WfaGpuError(rc, "wfa_gpu_align_batch")
        if score_only:
            return scores, status, np.zeros(0, np.uint32), offs
        return scores, status, words[: int(offs[n])], offs

    def align_device(self, pat, poff, plen, txt, toff, tlen, out_scores, out_status, out_cigars,
                     out_cigar_offsets, pen=(4, 6, 2), max_score: int = 0, score_only: bool = False,
                     timing: bool = False, plain: bool = False, graph: bool = False,
                     arena_only: bool = False) -> int:
        """Device-memory call on torch CUDA tensors (offsets may be None).
        Returns the raw code (WFA_GPU_OK or WFA_GPU_ECIGAR_CAPACITY; other
        codes raise)."""
        n = int(plen.numel())
        flags = WFA_GPU_DEVICE_PTRS | (WFA_GPU_SCORE_ONLY if score_only else 0) | \
            (WFA_GPU_TIMING if timing else 0) | (WFA_GPU_PLAIN if plain else 0) | (WFA_GPU_GRAPH if graph else 0) | \
            (WFA_GPU_ARENA_ONLY if arena_only else 0)
        cap = 0 if (score_only or out_cigars is None) else int(out_cigars.numel())
        rc = wfa_gpu_align_batch(self.ctx, n, _addr(pat), _addr(poff), _addr(plen), _addr(txt), _addr(toff),
                                 _addr(tlen), pen, max_score, flags, _addr(out_scores), _addr(out_status),
                                 _addr(out_cigars), cap, _addr(out_cigar_offsets))
        if rc not in (WFA_GPU_OK, WFA_GPU_ECIGAR_CAPACITY):
            raise WfaGpuError(rc, "wfa_gpu_align_batch")
        return rc

    def pack2bit(self, seqs: np.ndarray, offsets, lengths: np.ndarray):
        """Host-memory packer call.  Returns (words, word offsets, invalid)."""
        n = int(len(lengths))
        seqs = np.ascontiguousarray(seqs, dtype=np.uint8)
        lengths = np.ascontiguousarray(lengths, dtype=np.int32)
        offsets = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.int64)
        woff = np.zeros(n + 1, dtype=np.int64)
        inv = np.zeros(max(n, 1), dtype=np.int8)
        cap = int(((lengths.astype(np.int64) + 31) // 32 + 1).sum()) if n else 0
        words = np.zeros(max(cap, 1), dtype=np.uint64)
        rc = wfa_gpu_pack2bit(self.ctx, n, _addr(seqs), _addr(offsets), _addr(lengths), 0, _addr(words), cap,
                              _addr(woff), _addr(inv))
        if rc != WFA_GPU_OK:
            raise WfaGpuError(rc, "wfa_gpu_pack2bit")
        return words[:cap], woff, inv[:n]


# ------------------------------------------------------------------ serving


def wfa_gpu_server_create(device: int = 0, workers: int = 4, memory_budget_bytes: int = 0):
    h = ctypes.c_void_p()
    rc = load().wfa_gpu_server_create(ctypes.byref(h), device, workers, memory_budget_bytes)
    return rc, (h if rc == WFA_GPU_OK else None)


def wfa_gpu_server_submit(server, req: Request) -> int:
    return load().wfa_gpu_server_submit(server, ctypes.byref(req))


def wfa_gpu_server_wait(server, rid: int, timeout_s: float = -1.0):
    st = RequestStats()
    rc = load().wfa_gpu_server_wait(server, rid, timeout_s, ctypes.byref(st))
    return rc, st


def wfa_gpu_request_bytes(req: Request) -> int:
    return load().wfa_gpu_request_bytes(ctypes.byref(req))


def wfa_gpu_server_destroy(server) -> None:
    load().wfa_gpu_server_destroy(server)


class Server:
    """Continuous-batching request server (host buffers).  ``submit`` takes a
    batch and returns a request id at once; ``wait`` returns its outputs
    (scores, status, CIGAR words, CIGAR offsets) and timing."""

    def __init__(self, device: int = 0, workers: int = 4, memory_budget_bytes: int = 0):
        rc, h = wfa_gpu_server_create(device, workers, memory_budget_bytes)
        if rc != WFA_GPU_OK:
            raise WfaGpuError(rc, "wfa_gpu_server_create")
        self.h = h
        self._pending = {}

    def submit(self, batch, pen=(4, 6, 2), max_score: int = 0, score_only: bool = False, plain: bool = False,
               arena_only: bool = False,
               cigar_capacity: int | None = None) -> int:
        n = int(len(batch.pattern_lengths))
        keep = dict(
            pat=np.ascontiguousarray(batch.patterns, dtype=np.uint8),
            txt=np.ascontiguousarray(batch.texts, dtype=np.uint8),
            plen=np.ascontiguousarray(batch.pattern_lengths, dtype=np.int32),
            tlen=np.ascontiguousarray(batch.text_lengths, dtype=np.int32),
            poff=None if batch.pattern_offsets is None else np.ascontiguousarray(batch.pattern_offsets, np.int64),
            toff=None if batch.text_offsets is None else np.ascontiguousarray(batch.text_offsets, np.int64),
            s=np.empty(n, np.int32), st=np.empty(n, np.int8), off=np.zeros(n + 1, np.int64))
        if cigar_capacity is None:
            bound = sum(int(wfa_gpu_cigar_bound(int(p), int(t), pen, max_score))
                        for p, t in zip(keep["plen"], keep["tlen"])) if not score_only else 0
            cigar_capacity = bound
        keep["w"] = np.empty(max(1, cigar_capacity), np.uint32)
        flags = (WFA_GPU_SCORE_ONLY if score_only else 0) | (WFA_GPU_PLAIN if plain else 0) | \
            (WFA_GPU_ARENA_ONLY if arena_only else 0)
        req = Request(n, _addr(keep["pat"]), _addr(keep["poff"]), _addr(keep["plen"]), _addr(keep["txt"]),
                      _addr(keep["toff"]), _addr(keep["tlen"]), pen if isinstance(pen, Penalties) else Penalties(*pen),
                      max_score, flags, _addr(keep["s"]), _addr(keep["st"]), None if score_only else _addr(keep["w"]),
                      0 if score_only else cigar_capacity, None if score_only else _addr(keep["off"]))
        keep["req"] = req
        rid = wfa_gpu_server_submit(self.h, req)
        if rid < 0:
            raise WfaGpuError(int(rid), "wfa_gpu_server_submit")
        self._pending[rid] = keep
        return rid

    def wait(self, rid: int, timeout_s: float = -1.0, check: bool = True):
        """Outputs and stats of request ``rid``.  With ``check`` a result
        other than OK raises WfaGpuError; without it the outputs are returned
        as the call left them and ``stats.result`` holds the code."""
        rc, st = wfa_gpu_server_wait(self.h, rid, timeout_s)
        if rc == WFA_GPU_ETIMEOUT:
            raise TimeoutError("request %d still running" % rid)
        keep = self._pending.pop(rid)
        if rc != WFA_GPU_OK and check:
            raise WfaGpuError(rc, "request %d" % rid)
        off = keep["off"]
        used = int(off[-1]) if rc == WFA_GPU_OK else 0
        return (keep["s"], keep["st"], keep["w"][:used], off), st

    def close(self):
        if self.h is not None:
            wfa_gpu_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
