"""The C-ABI library builds for sm_103a, loads, and exports every function
include/wfa_gpu.h declares; host-only entry points behave as documented.
No compute call is made here (no GPU is needed)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wfa_gpu.h")


@pytest.fixture(scope="module")
def pkg():
    from paper_2204_02085_gb300 import build

    build.build()
    import paper_2204_02085_gb300 as p

    p.load()
    return p


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wfa_gpu_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("wfa_gpu_create", "wfa_gpu_align_batch", "wfa_gpu_destroy", "wfa_gpu_cigar_bound",
                     "wfa_gpu_strerror"):
        assert required in names


def test_exports_every_declared_symbol(pkg):
    lib = pkg.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(pkg.EXPORTS) == declared_functions()
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (wfa_gpu_\w+)", out))
    assert set(declared_functions()) <= exported


def test_library_targets_sm103a(pkg):
    from paper_2204_02085_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_strerror(pkg):
    for code in (0, -1, -2, -3, -4, -5, 12345):
        s = pkg.wfa_gpu_strerror(code)
        assert isinstance(s, str) and s
    assert pkg.wfa_gpu_strerror(-4).startswith("CIGAR")


def test_cigar_bound(pkg):
    pen = (4, 6, 2)
    assert pkg.wfa_gpu_cigar_bound(0, 0, pen, 0) == 0
    assert pkg.wfa_gpu_cigar_bound(-1, 5, pen, 0) == -1
    assert pkg.wfa_gpu_cigar_bound(5, 5, (0, 6, 2), 0) == -1
    assert pkg.wfa_gpu_cigar_bound(5, 5, (4, -1, 2), 0) == -1
    assert pkg.wfa_gpu_cigar_bound(5, 5, (4, 6, 0), 0) == -1
    # never more runs than columns
    assert pkg.wfa_gpu_cigar_bound(100, 100, pen, 0) <= 200
    # with a score bound: 2*floor(s/min(x, o+e)) + 1
    assert pkg.wfa_gpu_cigar_bound(100, 100, pen, 16) == 2 * (16 // 4) + 1
    assert pkg.wfa_gpu_cigar_bound(100, 100, (16, 6, 2), 16) == 2 * (16 // 8) + 1
    assert 1 <= pkg.wfa_gpu_cigar_bound(10, 0, pen, 0) <= 10


def test_cigar_bound_covers_oracle_alignments(pkg, oracle_mod):
    """The bound holds for every canonical alignment of random pairs."""
    from paper_2204_02085_gb300 import synth

    b = synth.random_pairs(200, 0, 60, seed=13)
    for pen in ((4, 6, 2), (1, 0, 1), (16, 6, 2), (2, 3, 1)):
        for i in range(b.n):
            p, t = b.pair(i)
            st, s, ops = oracle_mod.wfa(p, t, pen)
            runs = len(oracle_mod.ops_to_runs(ops))
            assert runs <= pkg.wfa_gpu_cigar_bound(len(p), len(t), pen, 0)
            assert runs <= pkg.wfa_gpu_cigar_bound(len(p), len(t), pen, s if s > 0 else 1) or s == 0


def test_null_arguments_rejected_without_device(pkg):
    lib = pkg.load()
    assert lib.wfa_gpu_create(None, 0, 0) == pkg.WFA_GPU_EINVAL
    h = ctypes.c_void_p()
    assert lib.wfa_gpu_create(ctypes.byref(h), -1, 0) == pkg.WFA_GPU_EINVAL
    assert pkg.wfa_gpu_align_batch(None, 1, None, None, None, None, None, None, (4, 6, 2), 0, 0, None, None,
                                   None, 0, None) == pkg.WFA_GPU_EINVAL
    assert pkg.wfa_gpu_set_stream(None, None) == pkg.WFA_GPU_EINVAL
    assert lib.wfa_gpu_last_timing(None, None) == pkg.WFA_GPU_EINVAL
    pkg.wfa_gpu_destroy(None)  # NULL-safe


def test_create_without_gpu_fails_cleanly(pkg):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, h = pkg.wfa_gpu_create(0, 0)
    assert rc == pkg.WFA_GPU_ECUDA and h is None


def test_product_never_imports_the_oracle():
    """The library package and the C sources do not reference oracle/."""
    pkg_dir = os.path.join(ROOT, "paper_2204_02085_gb300")
    for dirpath, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "wfa_oracle" not in text, f


def test_request_bytes_is_host_only(pkg):
    """The admission measure of the serving API: sequence bytes plus a fixed
    per-pair share, the caller's CIGAR capacity and the arena the wavefronts
    of pairs longer than 127 bases take; no device needed."""
    import numpy as np

    plen = np.array([100, 0, 250], np.int32)
    tlen = np.array([90, 10, 300], np.int32)
    req = pkg.Request(3, None, None, plen.ctypes.data, None, None, tlen.ctypes.data, pkg.Penalties(4, 6, 2), 0, 0,
                      None, None, None, 1000, None)
    # the third pair (300 bases) only: g = 2, costliest edit max(4, 6 + 2) / 2
    # = 4, e' = 1, s' = 0.10 x 300 x 4 = 120, (s'/e' + 1)^2 cells of 3
    # two-byte offsets, 16 bytes of metadata per score
    wavefront = int(3 * 2 * 121 ** 2 + 16 * 121)
    assert pkg.wfa_gpu_request_bytes(req) == int(plen.sum() + tlen.sum()) + 150 * 3 + 4 * 1000 + wavefront
    bad = pkg.Request(-1, None, None, None, None, None, None, pkg.Penalties(4, 6, 2), 0, 0, None, None, None, 0, None)
    assert pkg.wfa_gpu_request_bytes(bad) == -1
    assert pkg.load().wfa_gpu_server_create(None, 0, 4, 0) == pkg.WFA_GPU_EINVAL
    pkg.wfa_gpu_server_destroy(None)


def test_header_constants_match_binding():
    """Every integer #define and enum value of the header that the binding
    mirrors has the same value there."""
    import paper_2204_02085_gb300 as p

    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    seen = 0
    for name, expr in re.findall(r"#define\s+(WFA_GPU_[A-Z0-9_]+)\s+(.+)", text):
        if hasattr(p, name) and re.fullmatch(r"[()0-9<>\s\-+]*", expr.replace("(size_t)", "")):
            assert getattr(p, name) == eval(expr.replace("(size_t)", "")), name
            seen += 1
    for name, val in re.findall(r"\b(WFA_(?:GPU|PAIR)_[A-Z0-9_]+)\s*=\s*(-?\d+)", text):
        if hasattr(p, name):
            assert getattr(p, name) == int(val), name
            seen += 1
    assert seen >= 10
    assert p.WFA_GPU_SERVER_MERGE_PAIRS == 65536 and p.WFA_GPU_MAX_SEQ_LEN == (1 << 28) - 1


def test_missing_library_fails_loudly():
    """Without libwfa_gpu.so the binding raises at once: there is no CPU
    fallback behind the product API."""
    import subprocess
    import sys

    code = ("import paper_2204_02085_gb300 as p\n"
            "try:\n"
            "    p.load('/nonexistent/libwfa_gpu.so')\n"
            "except ImportError as e:\n"
            "    print('raised', 'not built' in str(e))\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == "raised True"


def _request(pkg, plens, tlens, pen=(4, 6, 2), cap=0):
    """A request carrying only what the byte estimate reads (host-only)."""
    import numpy as np

    p = np.ascontiguousarray(plens, dtype=np.int32)
    t = np.ascontiguousarray(tlens, dtype=np.int32)
    r = pkg.Request()
    r.n_pairs = len(p)
    r.pattern_lengths = p.ctypes.data if len(p) else None
    r.text_lengths = t.ctypes.data if len(t) else None
    r.pen = pkg.Penalties(*pen)
    r.cigar_capacity_words = cap
    return r, (p, t)  # the arrays must outlive the call


def test_request_bytes_closed_form(pkg):
    """wfa_gpu_request_bytes on hand-worked cases.  A request holds its
    sequence bytes, 150 bytes a pair, 4 per CIGAR word of capacity, and for
    each pair longer than 127 bases 3 offsets of 2 bytes (4 from 32,000
    bases) on (s'/e' + 1)^2 cells plus 16 (s' + 1) bytes, with
    s' = 0.10 * max(n, m) * max(x, o + e) / g, e' = e / g, g = gcd(x, o, e);
    over the 4,096 largest such pairs only."""
    rb = pkg.wfa_gpu_request_bytes
    # no pairs: the CIGAR capacity alone
    r, keep = _request(pkg, [], [], cap=7)
    assert rb(r) == 28
    # short pairs keep their wavefronts in shared memory: no arena term
    r, keep = _request(pkg, [100, 127], [100, 120], cap=10)
    assert rb(r) == (100 + 100 + 127 + 120) + 2 * 150 + 4 * 10
    # 1,000 bases under 4/6/2: g = 2, max(x, o + e) / g = 4, e' = 1,
    # s' = 0.10 * 1000 * 4 = 400: 3 * 2 * 401^2 + 16 * 401 = 971,222
    r, keep = _request(pkg, [1000], [990])
    assert rb(r) == 1990 + 150 + 971222
    # the longer sequence sets L; a negative length counts as 0 bytes
    r, keep = _request(pkg, [-5], [1000])
    assert rb(r) == 1000 + 150 + 971222
    # 40,000 bases: 4-byte offsets, s' = 16,000:
    # 3 * 4 * 16001^2 + 16 * 16001 = 3,072,640,028
    r, keep = _request(pkg, [40000], [40000])
    assert rb(r) == 80000 + 150 + 3072640028
    # other penalties: 2/3/1 has g = 1, max(x, o + e) = 4, e' = 1: the same
    # s' as 4/6/2 and the same bytes; 6/4/2 has g = 2, max = 6 / 2 = 3, e' = 1,
    # s' = 300: 3 * 2 * 301^2 + 16 * 301 = 548,422
    r, keep = _request(pkg, [1000], [1000], pen=(2, 3, 1))
    assert rb(r) == 2000 + 150 + 971222
    r, keep = _request(pkg, [1000], [1000], pen=(6, 4, 2))
    assert rb(r) == 2000 + 150 + 548422
    # 4,097 pairs of 200 bases and one of 300: only the 4,096 largest count
    # (the 300-base pair and 4,095 of the others).  200 bases: s' = 80,
    # 3 * 2 * 81^2 + 16 * 81 = 40,662; 300 bases: s' = 120,
    # 3 * 2 * 121^2 + 16 * 121 = 89,782
    r, keep = _request(pkg, [200] * 4097 + [300], [200] * 4097 + [300])
    assert rb(r) == (400 * 4097 + 600) + 150 * 4098 + 4095 * 40662 + 89782


def test_request_bytes_rejects_malformed(pkg):
    rb = pkg.wfa_gpu_request_bytes
    r, keep = _request(pkg, [10], [10])
    r.n_pairs = -1
    assert rb(r) == -1
    r, keep = _request(pkg, [10], [10])
    r.pattern_lengths = None
    assert rb(r) == -1
