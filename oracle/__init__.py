"""Plain CPU oracle for exact gap-affine pairwise alignment.

TEST INFRASTRUCTURE ONLY.  The library under test never imports, loads or
calls anything here.  The only callers are ``tests/``, the smoke check in
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``.

The arithmetic lives in ``wfa_oracle.c`` (plain C, compiled with gcc into
``liboracle.so`` beside it); this module only marshals arguments.  It shares
no code with the CUDA path: the two meet only at the seeded input generator
(``paper_2204_02085_gb300.synth``), which holds none of the method's
arithmetic.

Functions (each follows the paper's method, WFA, Sec. I, run unmodified):

* ``brute(p, t, pen)``      every alignment enumerated and rescored
* ``gotoh(p, t, pen)``      textbook O(nm) DP + walk-back traceback
* ``wfa(p, t, pen)``        the wavefront recurrences + backtrace
* ``rescore(p, t, ops, pen)``  the cost definition applied to one alignment
* ``pack2bit(seq)``         the 2-bit packed format (reference for the packer)
* ``wfa_batch(...)``        ``wfa`` over many pairs on POSIX threads

Penalties are ``(x, o, e)``: mismatch x, a gap run of length L costs o + L*e,
match 0.  ``ends`` = (pattern begin, pattern end, text begin, text end) free
lengths selects ends-free alignment (see ``wfa_oracle.c``); the default
(0, 0, 0, 0) is the global alignment.  Alignments are op strings over ``M X I D`` (I consumes text, D
consumes pattern) or run-length words ``(len << 4) | code`` with codes
M=0 X=1 I=2 D=3.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wfa_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, SCORE_LIMIT, INVALID_CHAR = 0, 1, 2
OP_CODES = {"M": 0, "X": 1, "I": 2, "D": 3}
OP_CHARS = "MXID"


class Counts(ctypes.Structure):
    _fields_ = [
        ("cells", ctypes.c_int64),
        ("wavefronts", ctypes.c_int64),
        ("char_compares", ctypes.c_int64),
        ("bt_steps", ctypes.c_int64),
    ]


def build(force: bool = False) -> str:
    """Compile wfa_oracle.c into liboracle.so for this machine."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC, "-lpthread"]
        )
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            i64, i32, cp = ctypes.c_int64, ctypes.c_int32, ctypes.c_char_p
            vp = ctypes.c_void_p
            L.oracle_valid.argtypes = [cp, i64]
            L.oracle_valid.restype = ctypes.c_int
            L.oracle_rescore_ef.argtypes = [cp, i64, cp, i64, cp, i64, i64, i64, i64, i64, i64, i64, i64]
            L.oracle_rescore_ef.restype = i64
            L.oracle_brute_ef.argtypes = [cp, ctypes.c_int, cp, ctypes.c_int, i64, i64, i64, i64, i64, i64, i64,
                                          vp, vp, vp]
            L.oracle_brute_ef.restype = i64
            L.oracle_gotoh_ef.argtypes = [cp, i64, cp, i64, i64, i64, i64, i64, i64, i64, i64, vp, vp]
            L.oracle_gotoh_ef.restype = i64
            L.oracle_wfa_ef.argtypes = [cp, i64, cp, i64, i64, i64, i64, i64, i64, i64, i64, i64, ctypes.c_int,
                                        vp, vp, i64, vp, vp]
            L.oracle_wfa_ef.restype = ctypes.c_int
            L.oracle_pack2bit.argtypes = [cp, i64, vp]
            L.oracle_pack2bit.restype = ctypes.c_int
            L.oracle_runs_encode.argtypes = [cp, i64, vp, i64]
            L.oracle_runs_encode.restype = i64
            L.oracle_wfa_batch_ef.argtypes = [i64, vp, vp, vp, vp, vp, vp, i64, i64, i64, i64, i64, i64, i64,
                                              i64, vp, vp, vp, i64, vp, ctypes.c_int, vp]
            L.oracle_wfa_batch_ef.restype = ctypes.c_int
            _lib = L
    return _lib


def _b(s) -> bytes:
    return s.encode() if isinstance(s, str) else bytes(s)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


GLOBAL = (0, 0, 0, 0)


def rescore(p, t, ops: str, pen, ends=GLOBAL) -> int:
    """Cost of alignment ``ops`` of p and t, or -1 if it is not one."""
    p, t, o = _b(p), _b(t), ops.encode()
    x, go, ge = pen
    return lib().oracle_rescore_ef(p, len(p), t, len(t), o, len(o), x, go, ge, *ends)


def brute(p, t, pen, ends=GLOBAL):
    """(minimum cost, canonical op string, number of alignments enumerated)."""
    p, t = _b(p), _b(t)
    x, go, ge = pen
    buf = ctypes.create_string_buffer(32)
    nops, npaths = ctypes.c_int64(), ctypes.c_int64()
    c = lib().oracle_brute_ef(p, len(p), t, len(t), x, go, ge, *ends, ctypes.cast(buf, ctypes.c_void_p),
                              ctypes.byref(nops), ctypes.byref(npaths))
    if c < 0:
        raise ValueError("brute force takes lengths <= 12")
    return c, buf.raw[: nops.value].decode(), npaths.value


def gotoh(p, t, pen, want_ops: bool = True, ends=GLOBAL):
    """(score, op string or None) from the Gotoh DP and its walk-back."""
    p, t = _b(p), _b(t)
    x, go, ge = pen
    if want_ops:
        buf = ctypes.create_string_buffer(len(p) + len(t) + 1)
        nops = ctypes.c_int64()
        s = lib().oracle_gotoh_ef(p, len(p), t, len(t), x, go, ge, *ends,
                                  ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(nops))
        if s < 0:
            raise RuntimeError("oracle_gotoh failed (%d)" % s)
        return s, buf.raw[: nops.value].decode()
    s = lib().oracle_gotoh_ef(p, len(p), t, len(t), x, go, ge, *ends, None, None)
    if s < 0:
        raise RuntimeError("oracle_gotoh failed (%d)" % s)
    return s, None


def wfa(p, t, pen, max_score: int = 0, want_ops: bool = True, counts: Counts | None = None, ends=GLOBAL):
    """(status, score, op string or None) from the CPU wavefront algorithm."""
    p, t = _b(p), _b(t)
    x, go, ge = pen
    score = ctypes.c_int64()
    cap = len(p) + len(t) + 1
    buf = ctypes.create_string_buffer(cap)
    nops = ctypes.c_int64()
    rc = lib().oracle_wfa_ef(p, len(p), t, len(t), x, go, ge, *ends, max_score, int(want_ops),
                             ctypes.byref(score), ctypes.cast(buf, ctypes.c_void_p), cap,
                             ctypes.byref(nops), ctypes.byref(counts) if counts is not None else None)
    if rc < 0:
        raise RuntimeError("oracle_wfa failed (%d)" % rc)
    ops = buf.raw[: nops.value].decode() if (want_ops and rc == OK) else None
    return rc, score.value if rc == OK else -1, ops


def pack2bit(seq) -> tuple[int, np.ndarray]:
    """(0 or -1 for an invalid byte, packed words: ceil(L/32) + 1 uint64)."""
    s = _b(seq)
    out = np.zeros((len(s) + 31) // 32 + 1, dtype=np.uint64)
    rc = lib().oracle_pack2bit(s, len(s), _ptr(out))
    return rc, out


def ops_to_runs(ops: str) -> list[int]:
    runs = []
    i = 0
    while i < len(ops):
        j = i
        while j < len(ops) and ops[j] == ops[i]:
            j += 1
        runs.append(((j - i) << 4) | OP_CODES[ops[i]])
        i = j
    return runs


def runs_to_ops(runs) -> str:
    return "".join(OP_CHARS[int(w) & 15] * (int(w) >> 4) for w in runs)


def runs_to_cigar(runs) -> str:
    return "".join("%d%s" % (int(w) >> 4, OP_CHARS[int(w) & 15]) for w in runs)


def wfa_batch(batch, pen, max_score: int = 0, want_cigar: bool = True,
              nthreads: int = 1, runs_per_pair: int | None = None, counts: Counts | None = None,
              ends=GLOBAL):
    """Align every pair of ``batch`` (a ``synth.Batch``-like object with
    patterns/pattern_offsets/pattern_lengths/texts/text_offsets/text_lengths)
    with the CPU WFA.  Returns (scores int32, status int8, cigar words uint32,
    cigar offsets int64 of length n+1)."""
    n = int(len(batch.pattern_lengths))
    pat = np.ascontiguousarray(batch.patterns, dtype=np.uint8)
    txt = np.ascontiguousarray(batch.texts, dtype=np.uint8)
    poff = np.ascontiguousarray(batch.pattern_offsets, dtype=np.int64)
    toff = np.ascontiguousarray(batch.text_offsets, dtype=np.int64)
    plen = np.ascontiguousarray(batch.pattern_lengths, dtype=np.int32)
    tlen = np.ascontiguousarray(batch.text_lengths, dtype=np.int32)
    scores = np.empty(n, dtype=np.int32)
    status = np.empty(n, dtype=np.int8)
    x, go, ge = pen
    if want_cigar:
        if runs_per_pair is None:
            runs_per_pair = int(max(1, (plen.max(initial=0) + tlen.max(initial=0)) if n else 1))
        runs = np.zeros(n * runs_per_pair, dtype=np.uint32)
        nruns = np.zeros(n, dtype=np.int32)
        rp, np_ = _ptr(runs), _ptr(nruns)
    else:
        runs_per_pair = 0
        runs = nruns = None
        rp = np_ = None
    rc = lib().oracle_wfa_batch_ef(n, _ptr(pat), _ptr(poff), _ptr(plen), _ptr(txt), _ptr(toff),
                                   _ptr(tlen), x, go, ge, *ends, max_score, _ptr(scores), _ptr(status),
                                   rp, runs_per_pair, np_, int(nthreads),
                                   ctypes.byref(counts) if counts is not None else None)
    if rc < 0:
        raise RuntimeError("oracle_wfa_batch failed (%d)" % rc)
    offsets = np.zeros(n + 1, dtype=np.int64)
    if not want_cigar:
        return scores, status, np.zeros(0, dtype=np.uint32), offsets
    np.cumsum(nruns, out=offsets[1:])
    words = np.empty(int(offsets[-1]), dtype=np.uint32)
    # gather each pair's runs into one contiguous array
    idx = np.repeat(np.arange(n, dtype=np.int64) * runs_per_pair - offsets[:-1], nruns)
    idx += np.arange(int(offsets[-1]), dtype=np.int64)
    words[:] = runs[idx]
    return scores, status, words, offsets
