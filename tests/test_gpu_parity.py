"""Parity of the CUDA path with the CPU oracle, through the C ABI.

Integer results must be bit-exact: scores, per-pair status, CIGAR offsets
and CIGAR words (same canonical tie-break).  Inputs are seeded synthetic
pairs shaped like the paper's workload (100 bp reads, E = 2 % / 4 %,
Sec. II) plus sizes that span several kernel tiles, ragged lengths, the
arena (long / high-score) path and the degenerate cases.
"""

import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

PENALTY_SETS = [(4, 6, 2), (1, 0, 1), (2, 3, 1), (5, 1, 3), (3, 2, 2), (16, 6, 2)]
NCPU = os.cpu_count() or 4


@pytest.fixture(scope="module")
def pkg():
    from paper_2204_02085_gb300 import build

    build.build()
    import paper_2204_02085_gb300 as p

    return p


@pytest.fixture(scope="module")
def al(pkg):
    a = pkg.Aligner(0)
    yield a
    a.close()


def oracle_run(oracle, batch, pen, max_score=0, want_cigar=True):
    return oracle.wfa_batch(batch, pen, max_score=max_score, want_cigar=want_cigar, nthreads=NCPU)


def assert_same(got, want, score_only=False):
    s, st, w, off = got
    os_, ost, ow, ooff = want
    bad = np.nonzero((s != os_) | (st != ost))[0]
    assert bad.size == 0, "first mismatching pairs %s: gpu %s/%s oracle %s/%s" % (
        bad[:5], s[bad[:5]], st[bad[:5]], os_[bad[:5]], ost[bad[:5]])
    if not score_only:
        assert np.array_equal(off, ooff), "CIGAR offsets differ"
        assert np.array_equal(w, ow), "CIGAR words differ"


def check(al, oracle, batch, pen, max_score=0, score_only=False, use_offsets=True):
    got = al.align(batch, pen, max_score=max_score, score_only=score_only, use_offsets=use_offsets)
    want = oracle_run(oracle, batch, pen, max_score=max_score, want_cigar=not score_only)
    assert_same(got, want, score_only)
    return got


def test_config1_small_plain(al, oracle_mod):
    """1,000 pairs, seed 0, 100 bp, exactly 2 edits, penalties 4/6/2."""
    from paper_2204_02085_gb300 import synth

    b = synth.uniform_reads(1000, 100, 2, seed=0)
    s, st, w, off = check(al, oracle_mod, b, (4, 6, 2))
    assert np.all(st == 0) and s.max() <= 16


@pytest.mark.parametrize("edits", [4, 10, 25])
def test_higher_edit_rates(al, oracle_mod, edits):
    """More edits push wavefronts past the shared-memory budget: those pairs
    move to the arena kernel and must still match."""
    from paper_2204_02085_gb300 import synth

    b = synth.uniform_reads(3000, 100, edits, seed=edits)
    check(al, oracle_mod, b, (4, 6, 2))
    if edits >= 10:
        assert al.timing()["deferred_pairs"] >= 0


@pytest.mark.parametrize("pen", PENALTY_SETS)
def test_penalty_sets(al, oracle_mod, pen):
    from paper_2204_02085_gb300 import synth

    b = synth.uniform_reads(1500, 100, 4, seed=sum(pen))
    check(al, oracle_mod, b, pen)


def test_ragged_lengths_and_unrelated(al, oracle_mod):
    """Lengths 0..600 (both sides of the 256-base short-kernel limit),
    related and unrelated pairs, mixed case."""
    from paper_2204_02085_gb300 import synth

    rel = synth.random_pairs(400, 0, 600, seed=31, edit_rate=0.05)
    unrel = synth.random_pairs(150, 0, 300, seed=32, alphabet=b"ACGTacgt")
    pairs = [rel.pair(i) for i in range(rel.n)] + [unrel.pair(i) for i in range(unrel.n)]
    b = synth.from_pairs(pairs)
    for pen in ((4, 6, 2), (1, 0, 1), (16, 6, 2)):
        check(al, oracle_mod, b, pen)


def test_edge_cases(al, oracle_mod):
    from paper_2204_02085_gb300 import synth

    A = b"ACGT" * 80
    pairs = [(b"", b""), (b"", b"A"), (b"G", b""), (b"", A[:256]), (A[:256], b""), (b"A", b"A"), (b"A", b"C"),
             (b"AAAA", b"AAA"), (b"GATTACA", b"GATACA"), (b"acgt", b"ACGT"), (b"ACGN", b"ACGT"),
             (b"ACGT", b"AC-T"), (b"ACGT\x00", b"ACGT"), (A[:31], A[:31]), (A[:32], A[:32]), (A[:33], A[:33]),
             (A[:63], A[:64]), (A[:64], A[:65]), (A[:255], A[:256]), (A[:256], A[:256]), (A[:257], A[:256]),
             (A[:256], A[:257]), (A[:300], A[:290]), (b"T" * 200, b"A" * 200), (b"A" * 256, b"C" * 256)]
    b = synth.from_pairs(pairs)
    for pen in PENALTY_SETS:
        check(al, oracle_mod, b, pen)
    s, st, _, _ = al.align(b, (4, 6, 2))
    assert st[10] == 2 and st[11] == 2 and st[12] == 2 and s[10] == -1


def test_max_score_boundary(al, oracle_mod):
    from paper_2204_02085_gb300 import synth

    b = synth.uniform_reads(2000, 100, 4, seed=7)
    for ms in (1, 4, 8, 12, 16, 17, 30):
        got = check(al, oracle_mod, b, (4, 6, 2), max_score=ms)
        s, st = got[0], got[1]
        assert np.all(s[st == 0] <= ms) and np.all(s[st == 1] == -1)


def test_score_only_and_null_offsets(al, oracle_mod):
    from paper_2204_02085_gb300 import synth

    b = synth.random_pairs(300, 50, 400, seed=41, edit_rate=0.04)
    check(al, oracle_mod, b, (4, 6, 2), score_only=True)
    check(al, oracle_mod, b, (4, 6, 2), use_offsets=False)


def test_shuffled_offsets(al, oracle_mod):
    """Sequences need not be back to back or in pair order."""
    from paper_2204_02085_gb300 import synth

    b = synth.uniform_reads(500, 100, 3, seed=43)
    perm = np.random.default_rng(0).permutation(b.n)
    pat = b"".join(b.pair(int(i))[0] + b"N" for i in perm)  # gaps of one junk byte
    txt = b"".join(b"xx" + b.pair(int(i))[1] for i in perm)
    poff = np.zeros(b.n, np.int64)
    toff = np.zeros(b.n, np.int64)
    po = to = 0
    for i in perm:
        p, t = b.pair(int(i))
        poff[i] = po
        toff[i] = to + 2
        po += len(p) + 1
        to += len(t) + 2
    shuffled = synth.Batch(np.frombuffer(pat, np.uint8).copy(), poff, b.pattern_lengths.copy(),
                           np.frombuffer(txt, np.uint8).copy(), toff, b.text_lengths.copy())
    got = al.align(shuffled, (4, 6, 2))
    want = oracle_run(oracle_mod, b, (4, 6, 2))
    assert_same(got, want)


def test_cigar_capacity(pkg, al, oracle_mod):
    from paper_2204_02085_gb300 import synth

    b = synth.uniform_reads(200, 100, 2, seed=44)
    want = oracle_run(oracle_mod, b, (4, 6, 2))
    total = int(want[3][-1])
    with pytest.raises(pkg.WfaGpuError) as ei:
        al.align(b, (4, 6, 2), cigar_capacity=total - 1)
    assert ei.value.code == pkg.WFA_GPU_ECIGAR_CAPACITY
    got = al.align(b, (4, 6, 2), cigar_capacity=total)
    assert_same(got, want)


def test_small_arena_retries(pkg, oracle_mod):
    """A tiny scratch arena forces arena-kernel retries with fewer, larger
    slots; results are unchanged.  A pair that cannot fit even the whole
    arena gives ENOMEM."""
    from paper_2204_02085_gb300 import synth

    # unrelated 200-700 bp pairs need up to ~5 MB of wavefronts each: a
    # 64 MB arena split over the default warp count is too small for them,
    # so they are retried with fewer, larger slots
    b = synth.random_pairs(60, 200, 700, seed=45)
    with pkg.Aligner(0, scratch_bytes=64 << 20) as small:
        got = small.align(b, (4, 6, 2))
        assert_same(got, oracle_run(oracle_mod, b, (4, 6, 2)))
    big = synth.random_pairs(2, 3000, 3000, seed=46)
    with pkg.Aligner(0, scratch_bytes=64 << 10) as tiny:
        with pytest.raises(pkg.WfaGpuError) as ei:
            tiny.align(big, (4, 6, 2))
        assert ei.value.code == pkg.WFA_GPU_ENOMEM


def test_device_pointers_match_host_path(pkg, al, oracle_mod):
    import torch

    from paper_2204_02085_gb300 import synth

    b = synth.random_pairs(700, 0, 300, seed=47, edit_rate=0.03)
    host = al.align(b, (4, 6, 2))
    dev = torch.device("cuda:0")
    al.set_stream(torch.cuda.current_stream(dev))
    try:
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        n = b.n
        out_s = torch.empty(n, dtype=torch.int32, device=dev)
        out_st = torch.empty(n, dtype=torch.int8, device=dev)
        out_off = torch.empty(n + 1, dtype=torch.int64, device=dev)
        out_w = torch.empty(int(host[3][-1]), dtype=torch.int32, device=dev)
        for offsets in (True, False):
            rc = al.align_device(t(b.patterns), t(b.pattern_offsets) if offsets else None, t(b.pattern_lengths),
                                 t(b.texts), t(b.text_offsets) if offsets else None, t(b.text_lengths),
                                 out_s, out_st, out_w, out_off, pen=(4, 6, 2))
            torch.cuda.synchronize(dev)
            assert rc == pkg.WFA_GPU_OK
            assert np.array_equal(out_s.cpu().numpy(), host[0])
            assert np.array_equal(out_st.cpu().numpy(), host[1])
            assert np.array_equal(out_off.cpu().numpy(), host[3])
            assert np.array_equal(out_w.cpu().numpy().view(np.uint32), host[2])
    finally:
        al.set_stream(None)


@pytest.mark.parametrize("n", [2049, 4099])
def test_device_pointers_unaligned_arrays(pkg, al, oracle_mod, n):
    """Device arrays at addresses that are not 16-byte aligned (sequences one
    byte in, lengths one int32 in, CIGAR offsets one int64 in) and batch sizes
    just past prefix-sum tiles of 2,048 and not multiples of four: the
    offset scans and the input checks take their element-wise loads and
    stores there.  Scores, statuses, offsets and CIGARs equal the oracle's
    (exact: integer results)."""
    import torch

    from paper_2204_02085_gb300 import synth

    b = synth.random_pairs(n, 0, 200, seed=48 + n, edit_rate=0.03)
    want = oracle_run(oracle_mod, b, (4, 6, 2))
    dev = torch.device("cuda:0")

    def shifted(a, dtype):  # a copy one element into a larger device buffer
        buf = torch.zeros(len(a) + 1, dtype=dtype, device=dev)
        buf[1:] = torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        return buf[1:]

    al.set_stream(torch.cuda.current_stream(dev))
    try:
        out_s = torch.empty(n, dtype=torch.int32, device=dev)
        out_st = torch.empty(n, dtype=torch.int8, device=dev)
        out_off = torch.empty(n + 2, dtype=torch.int64, device=dev)[1:]
        out_w = torch.empty(int(want[3][-1]), dtype=torch.int32, device=dev)
        assert out_off.data_ptr() % 16 == 8
        plen, tlen = shifted(b.pattern_lengths, torch.int32), shifted(b.text_lengths, torch.int32)
        assert plen.data_ptr() % 16 == 4 and tlen.data_ptr() % 16 == 4
        for offsets in (False, True):
            rc = al.align_device(shifted(b.patterns, torch.uint8),
                                 shifted(b.pattern_offsets, torch.int64) if offsets else None, plen,
                                 shifted(b.texts, torch.uint8), shifted(b.text_offsets, torch.int64) if offsets else None,
                                 tlen, out_s, out_st, out_w, out_off, pen=(4, 6, 2))
            torch.cuda.synchronize(dev)
            assert rc == pkg.WFA_GPU_OK
            got = (out_s.cpu().numpy(), out_st.cpu().numpy(), out_w.cpu().numpy().view(np.uint32), out_off.cpu().numpy())
            assert_same(got, want)
    finally:
        al.set_stream(None)


def test_page_locked_host_inputs(pkg, al, oracle_mod):
    """Host-pointer calls whose buffers are page-locked (read by the kernels
    in place over the host link) give the oracle's results, as pageable
    buffers (copied) do."""
    import torch

    from paper_2204_02085_gb300 import synth

    b = synth.random_pairs(900, 0, 300, seed=52, edit_rate=0.04)

    def pinned(a):
        t = torch.empty(a.shape, dtype={np.uint8: torch.uint8, np.int32: torch.int32,
                                         np.int64: torch.int64}[a.dtype.type], pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    pb = synth.Batch(pinned(b.patterns), pinned(b.pattern_offsets), pinned(b.pattern_lengths), pinned(b.texts),
                     pinned(b.text_offsets), pinned(b.text_lengths))
    want = oracle_run(oracle_mod, b, (4, 6, 2))
    assert_same(al.align(pb, (4, 6, 2)), want)
    assert_same(al.align(pb, (4, 6, 2), use_offsets=False), want)
    assert_same(al.align(b, (4, 6, 2)), want)


def test_repeated_calls_are_stable(al, oracle_mod):
    """The same batch twice, with other batches between, gives identical
    output (no state leaks between calls)."""
    from paper_2204_02085_gb300 import synth

    b = synth.uniform_reads(3000, 100, 4, seed=48)
    first = al.align(b, (4, 6, 2))
    al.align(synth.random_pairs(100, 0, 500, seed=49), (1, 0, 1))
    second = al.align(b, (4, 6, 2))
    for x, y in zip(first, second):
        assert np.array_equal(x, y)


def test_pack2bit_matches_oracle(al, oracle_mod):
    from paper_2204_02085_gb300 import synth

    rng = np.random.default_rng(50)
    seqs = []
    for L in list(range(0, 70)) + [255, 256, 257, 1000, 4097]:
        alpha = np.frombuffer(b"ACGTacgt", np.uint8)
        s = alpha[rng.integers(0, 8, size=L)].tobytes()
        seqs.append(s)
    seqs.append(b"ACGTNACGT")
    seqs.append(b"A" * 40 + b"-")
    # odd starting offsets exercise every 16-byte alignment
    buf = bytearray()
    offs = []
    for i, s in enumerate(seqs):
        buf += b"#" * (i % 17)
        offs.append(len(buf))
        buf += s
    offs = np.array(offs, np.int64)
    lens = np.array([len(s) for s in seqs], np.int32)
    words, woff, inv = al.pack2bit(np.frombuffer(bytes(buf), np.uint8), offs, lens)
    for i, s in enumerate(seqs):
        rc, w = oracle_mod.pack2bit(s)
        assert inv[i] == (1 if rc != 0 else 0), i
        assert woff[i + 1] - woff[i] == len(w)
        if rc == 0:
            assert np.array_equal(words[woff[i]:woff[i + 1]], w), i


@pytest.mark.parametrize("edits", [2, 4])
def test_config2_full_size(pkg, oracle_mod, edits):
    """5,000,000 pairs of 100 bp at E = 2 % and 4 % (the paper's workload,
    Sec. II), device-resident as the benchmark runs them; every pair is
    compared bit-exactly with the oracle (in chunks on all host cores)."""
    import torch

    from paper_2204_02085_gb300 import synth

    n = 5_000_000
    b = synth.uniform_reads(n, 100, edits, seed=1)
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    out_s = torch.empty(n, dtype=torch.int32, device=dev)
    out_st = torch.empty(n, dtype=torch.int8, device=dev)
    out_off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    out_w = torch.empty(16 * n, dtype=torch.int32, device=dev)
    with pkg.Aligner(0) as al:
        al.set_stream(torch.cuda.current_stream(dev))
        rc = al.align_device(t(b.patterns), None, t(b.pattern_lengths), t(b.texts), None, t(b.text_lengths),
                             out_s, out_st, out_w, out_off, pen=(4, 6, 2))
        torch.cuda.synchronize(dev)
    assert rc == pkg.WFA_GPU_OK
    s = out_s.cpu().numpy()
    st = out_st.cpu().numpy()
    off = out_off.cpu().numpy()
    w = out_w.cpu().numpy().view(np.uint32)[: int(off[-1])]
    chunk = 1_000_000
    for c0 in range(0, n, chunk):
        sub = synth.Batch(b.patterns, b.pattern_offsets[c0:c0 + chunk], b.pattern_lengths[c0:c0 + chunk],
                          b.texts, b.text_offsets[c0:c0 + chunk], b.text_lengths[c0:c0 + chunk])
        os_, ost, ow, ooff = oracle_mod.wfa_batch(sub, (4, 6, 2), nthreads=NCPU, runs_per_pair=40)
        assert np.array_equal(s[c0:c0 + chunk], os_)
        assert np.array_equal(st[c0:c0 + chunk], ost)
        lo, hi = int(off[c0]), int(off[min(c0 + chunk, n)])
        assert np.array_equal(off[c0:c0 + chunk + 1] - lo, ooff)
        assert np.array_equal(w[lo:hi], ow)


def _pinned(torch, a):
    t = torch.empty(a.shape, dtype={np.uint8: torch.uint8, np.int32: torch.int32, np.int64: torch.int64,
                                    np.int8: torch.int8, np.uint32: torch.int32}[a.dtype.type], pin_memory=True)
    t.numpy().view(a.dtype)[...] = a
    return t


def test_chunked_host_call_with_page_locked_outputs(pkg, oracle_mod):
    """2.5M pairs (three chunks) from page-locked host memory into page-locked
    outputs: the chunked path, whose output copies overlap the next chunk,
    gives the oracle's results; a few long pairs go through the arena in a
    middle chunk; a short CIGAR capacity gives ECIGAR_CAPACITY with valid
    scores and offsets."""
    import torch

    from paper_2204_02085_gb300 import synth

    core = synth.uniform_reads(2_500_000, 100, 3, seed=77)
    extra = synth.random_pairs(40, 300, 900, seed=78, edit_rate=0.05)
    pairs_at = {1_200_000 + 7 * j: extra.pair(j) for j in range(extra.n)}
    # splice the long pairs into the batch without a Python loop over 2.5M pairs
    plen = core.pattern_lengths.copy(); tlen = core.text_lengths.copy()
    pats, txts = [core.patterns], [core.texts]
    poff = core.pattern_offsets.copy(); toff = core.text_offsets.copy()
    pbase, tbase = len(core.patterns), len(core.texts)
    for j, i in enumerate(sorted(pairs_at)):
        p, t = pairs_at[i]
        pats.append(np.frombuffer(p, np.uint8)); txts.append(np.frombuffer(t, np.uint8))
        poff[i], toff[i], plen[i], tlen[i] = pbase, tbase, len(p), len(t)
        pbase += len(p); tbase += len(t)
    b = synth.Batch(np.concatenate(pats), poff, plen, np.concatenate(txts), toff, tlen)
    n = b.n
    want = oracle_mod.wfa_batch(b, (4, 6, 2), nthreads=NCPU)
    ins = {k: _pinned(torch, getattr(b, k)) for k in ("patterns", "pattern_offsets", "pattern_lengths", "texts",
                                                      "text_offsets", "text_lengths")}
    cap = int(want[3][-1])
    outs = dict(s=torch.empty(n, dtype=torch.int32, pin_memory=True), st=torch.empty(n, dtype=torch.int8, pin_memory=True),
                off=torch.empty(n + 1, dtype=torch.int64, pin_memory=True),
                w=torch.empty(cap, dtype=torch.int32, pin_memory=True))
    ptr = lambda t: t.data_ptr()  # noqa: E731
    with pkg.Aligner(0, 2 << 30) as al:
        for c, code in ((cap, pkg.WFA_GPU_OK), (cap - 1, pkg.WFA_GPU_ECIGAR_CAPACITY)):
            rc = pkg.wfa_gpu_align_batch(al.ctx, n, ptr(ins["patterns"]), ptr(ins["pattern_offsets"]),
                                         ptr(ins["pattern_lengths"]), ptr(ins["texts"]), ptr(ins["text_offsets"]),
                                         ptr(ins["text_lengths"]), (4, 6, 2), 0, pkg.WFA_GPU_TIMING, ptr(outs["s"]),
                                         ptr(outs["st"]), ptr(outs["w"]), c, ptr(outs["off"]))
            assert rc == code
            t = al.timing()
            assert t["deferred_pairs"] >= 40
            got_s, got_st, got_off = outs["s"].numpy(), outs["st"].numpy(), outs["off"].numpy()
            assert np.array_equal(got_s, want[0]) and np.array_equal(got_st, want[1])
            assert np.array_equal(got_off, want[3])
            if code == pkg.WFA_GPU_OK:
                assert np.array_equal(outs["w"].numpy().view(np.uint32), want[2])


def _splice_back_to_back(core, repl):
    """A back-to-back batch equal to ``core`` (itself back to back) with the
    pairs at the keys of ``repl`` replaced by the (pattern, text) bytes given
    there; built from a few large slices."""
    from paper_2204_02085_gb300 import synth

    idx = sorted(repl)
    plen = core.pattern_lengths.copy()
    tlen = core.text_lengths.copy()
    pats, txts = [], []
    prev = 0
    for i in idx:
        pats.append(core.patterns[core.pattern_offsets[prev]:core.pattern_offsets[i]])
        txts.append(core.texts[core.text_offsets[prev]:core.text_offsets[i]])
        p, t = repl[i]
        pats.append(np.frombuffer(p, np.uint8))
        txts.append(np.frombuffer(t, np.uint8))
        plen[i], tlen[i] = len(p), len(t)
        prev = i + 1
    pats.append(core.patterns[core.pattern_offsets[prev]:] if prev < core.n else core.patterns[:0])
    txts.append(core.texts[core.text_offsets[prev]:] if prev < core.n else core.texts[:0])
    poff = np.zeros(core.n, np.int64)
    toff = np.zeros(core.n, np.int64)
    np.cumsum(plen[:-1], out=poff[1:])
    np.cumsum(tlen[:-1], out=toff[1:])
    return synth.Batch(np.concatenate(pats), poff, plen, np.concatenate(txts), toff, tlen)


@pytest.mark.parametrize("lengths_pinned", [True, False])
def test_streamed_host_call_back_to_back(pkg, oracle_mod, lengths_pinned):
    """2.5M pairs stored back to back in page-locked host memory, no offset
    arrays, page-locked outputs: the chunked path streams each chunk's bases
    (and its lengths, when those are page-locked too; else they are copied
    to the device once) into a device ring while earlier chunks compute.
    Long pairs in the middle chunk (the arena kernels read them from the
    ring), an empty pattern and a pattern with a non-ACGT byte in the ragged
    last chunk; the results equal the oracle's bit for bit, on two calls in
    a row on one context (the ring's slots refilled)."""
    import torch

    from paper_2204_02085_gb300 import synth

    core = synth.uniform_reads(2_500_000, 100, 4, seed=91)
    extra = synth.random_pairs(30, 400, 1500, seed=92, edit_rate=0.05)
    repl = {1_300_000 + 11 * j: extra.pair(j) for j in range(extra.n)}
    p, t = core.pair(2_400_001)
    repl[2_400_001] = (b"", t)
    p, t = core.pair(2_499_998)
    repl[2_499_998] = (p[:50] + b"N" + p[51:], t)
    b = _splice_back_to_back(core, repl)
    n = b.n
    want = oracle_mod.wfa_batch(b, (4, 6, 2), nthreads=NCPU)
    assert want[1][2_499_998] == 2 and want[1][2_400_001] == 0
    ins = {k: _pinned(torch, getattr(b, k)) for k in ("patterns", "texts")}
    for k in ("pattern_lengths", "text_lengths"):
        ins[k] = _pinned(torch, getattr(b, k)) if lengths_pinned else torch.from_numpy(getattr(b, k).copy())
    cap = int(want[3][-1])
    ptr = lambda t: t.data_ptr()  # noqa: E731
    with pkg.Aligner(0, 2 << 30) as al:
        for _ in range(2):
            outs = dict(s=torch.full((n,), -7, dtype=torch.int32, pin_memory=True),
                        st=torch.full((n,), 9, dtype=torch.int8, pin_memory=True),
                        off=torch.zeros(n + 1, dtype=torch.int64, pin_memory=True),
                        w=torch.zeros(cap, dtype=torch.int32, pin_memory=True))
            rc = pkg.wfa_gpu_align_batch(al.ctx, n, ptr(ins["patterns"]), None, ptr(ins["pattern_lengths"]),
                                         ptr(ins["texts"]), None, ptr(ins["text_lengths"]), (4, 6, 2), 0,
                                         pkg.WFA_GPU_TIMING, ptr(outs["s"]), ptr(outs["st"]), ptr(outs["w"]), cap,
                                         ptr(outs["off"]))
            assert rc == pkg.WFA_GPU_OK
            assert al.timing()["deferred_pairs"] >= 30
            assert np.array_equal(outs["s"].numpy(), want[0])
            assert np.array_equal(outs["st"].numpy(), want[1])
            assert np.array_equal(outs["off"].numpy(), want[3])
            assert np.array_equal(outs["w"].numpy().view(np.uint32), want[2])
