"""Serving with continuous batching: requests of mixed sizes submitted
together run concurrently on several slots, and every request's results are
bit-identical to aligning it alone (tolerance: exact; pairs are
independent, paper Sec. I)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2204_02085_gb300 import build

    build.build()
    import paper_2204_02085_gb300 as p

    return p


def _requests(seed, count):
    from paper_2204_02085_gb300 import synth

    rng = np.random.default_rng(seed)
    pool = synth.mixed_reads(3000, 100, 3000, 0.08, 0.05, seed=seed)
    short = synth.uniform_reads(4000, 100, 2, seed=seed + 1)
    reqs = []
    for j in range(count):
        size = int(np.exp(rng.uniform(0, np.log(1500))))
        src = short if j % 3 == 0 else pool
        start = int(rng.integers(0, src.n - size))
        reqs.append(synth.from_pairs([src.pair(i) for i in range(start, start + size)]))
    return reqs


def _overlaps(stats):
    iv = sorted((s.start_s, s.end_s) for s in stats)
    return sum(1 for a, b in zip(iv, iv[1:]) if b[0] < a[1])


def test_mix_equals_alone(pkg, oracle_mod):
    reqs = _requests(100, 24)
    with pkg.Aligner(0, 4 << 30) as al:
        alone = [al.align(b, (4, 6, 2)) for b in reqs]
    with pkg.Server(0, workers=4, memory_budget_bytes=16 << 30) as srv:
        ids = [srv.submit(b, (4, 6, 2), cigar_capacity=int(b.pattern_lengths.sum() + b.text_lengths.sum()) + 1)
               for b in reqs]
        outs = [srv.wait(i) for i in ids]
    stats = [st for _, st in outs]
    assert _overlaps(stats) > 0, "the requests never overlapped"
    assert len({st.worker for st in stats}) > 1
    for (got, st), want in zip(outs, alone):
        assert st.result == pkg.WFA_GPU_OK and st.submit_s <= st.start_s <= st.end_s
        for x, y in zip(got, want):
            assert np.array_equal(x, y)
    # and the oracle agrees on a few of them
    for j in (0, 1, 5):
        o = oracle_mod.wfa_batch(reqs[j], (4, 6, 2), nthreads=8)
        assert np.array_equal(outs[j][0][0], o[0]) and np.array_equal(outs[j][0][2], o[2])


def test_score_only_and_plain_requests(pkg):
    reqs = _requests(200, 6)
    with pkg.Aligner(0, 2 << 30) as al:
        alone = [al.align(b, (4, 6, 2), score_only=True) for b in reqs]
    with pkg.Server(0, workers=3, memory_budget_bytes=8 << 30) as srv:
        ids = [srv.submit(b, (4, 6, 2), score_only=True, plain=(j % 2 == 1)) for j, b in enumerate(reqs)]
        for rid, want in zip(ids, alone):
            (s, st, _, _), stats = srv.wait(rid)
            assert np.array_equal(s, want[0]) and np.array_equal(st, want[1])


def test_tiny_budget_admits_one_at_a_time(pkg):
    """With an arena no larger than one call's smallest slice (64 MiB), a
    call starts only when nothing else runs: no two calls overlap, results
    unchanged."""
    reqs = _requests(300, 8)
    with pkg.Aligner(0, 2 << 30) as al:
        alone = [al.align(b, (4, 6, 2)) for b in reqs]
    with pkg.Server(0, workers=4, memory_budget_bytes=64 << 20) as srv:
        ids = [srv.submit(b, (4, 6, 2), cigar_capacity=int(b.pattern_lengths.sum() + b.text_lengths.sum()) + 1)
               for b in reqs]
        outs = [srv.wait(i) for i in ids]
    # requests merged into one call share its interval: compare the calls
    calls = {(st.worker, st.start_s): st for _, st in outs}
    assert _overlaps(list(calls.values())) == 0
    for (got, _), want in zip(outs, alone):
        for x, y in zip(got, want):
            assert np.array_equal(x, y)


def test_wait_timeout_and_unknown_id(pkg):
    reqs = _requests(400, 1)
    with pkg.Server(0, workers=1) as srv:
        assert pkg.wfa_gpu_server_wait(srv.h, 12345, 0.0)[0] == pkg.WFA_GPU_EINVAL
        rid = srv.submit(reqs[0], (4, 6, 2))
        out, st = srv.wait(rid)
        assert st.result == pkg.WFA_GPU_OK


def _cap(b):
    return int(b.pattern_lengths.sum() + b.text_lengths.sum()) + 1


def test_merged_requests_equal_alone(pkg, oracle_mod):
    """One slot, many requests queued at once: the slot merges the ones that
    share parameters into one call, and every request still gets exactly its
    alone outputs."""
    reqs = _requests(500, 30)
    with pkg.Aligner(0, 4 << 30) as al:
        alone = [al.align(b, (4, 6, 2)) for b in reqs]
    with pkg.Server(0, workers=1, memory_budget_bytes=16 << 30) as srv:
        ids = [srv.submit(b, (4, 6, 2), cigar_capacity=_cap(b)) for b in reqs]
        outs = [srv.wait(i) for i in ids]
    stats = [st for _, st in outs]
    calls = {(st.worker, st.start_s) for st in stats}
    assert len(calls) < len(reqs), "no request was merged"
    for (got, st), want in zip(outs, alone):
        assert st.result == pkg.WFA_GPU_OK
        for x, y in zip(got, want):
            assert np.array_equal(x, y)
    o = oracle_mod.wfa_batch(reqs[7], (4, 6, 2), nthreads=8)
    assert np.array_equal(outs[7][0][0], o[0]) and np.array_equal(outs[7][0][2], o[2])


def test_merge_boundaries_and_errors(pkg):
    """A queue mixing what may and may not be merged: other penalties,
    score-only, plain, an empty request, a malformed one (negative length:
    EINVAL for it alone), one whose CIGAR capacity is too small
    (ECIGAR_CAPACITY with valid offsets, as alone), and sequences given
    without offset arrays.  Every request gets its alone result."""
    from paper_2204_02085_gb300 import synth

    reqs = _requests(600, 12)
    bad = synth.Batch(reqs[3].patterns, reqs[3].pattern_offsets, reqs[3].pattern_lengths.copy(), reqs[3].texts,
                      reqs[3].text_offsets, reqs[3].text_lengths)
    bad.pattern_lengths[min(2, bad.n - 1)] = -1
    empty = synth.from_pairs([])
    plan = []  # (batch, pen, kwargs, expected code)
    for j, b in enumerate(reqs):
        pen = (4, 6, 2) if j % 4 else (2, 3, 1)
        plan.append((b, pen, dict(cigar_capacity=_cap(b)), pkg.WFA_GPU_OK))
    plan.insert(2, (empty, (4, 6, 2), dict(cigar_capacity=0), pkg.WFA_GPU_OK))
    plan.insert(5, (bad, (4, 6, 2), dict(cigar_capacity=_cap(reqs[3]) + 10), pkg.WFA_GPU_EINVAL))
    plan.insert(6, (reqs[5], (4, 6, 2), dict(cigar_capacity=3), pkg.WFA_GPU_ECIGAR_CAPACITY))
    plan.insert(8, (reqs[6], (4, 6, 2), dict(score_only=True), pkg.WFA_GPU_OK))
    plan.insert(9, (reqs[7], (4, 6, 2), dict(score_only=True, plain=True), pkg.WFA_GPU_OK))
    plan.insert(10, (reqs[8], (4, 6, 2), dict(cigar_capacity=_cap(reqs[8]), plain=True), pkg.WFA_GPU_OK))
    packed = synth.from_pairs([reqs[9].pair(i) for i in range(reqs[9].n)])
    nooff = synth.Batch(packed.patterns, None, packed.pattern_lengths, packed.texts, None, packed.text_lengths)
    plan.insert(11, (nooff, (4, 6, 2), dict(cigar_capacity=_cap(packed)), pkg.WFA_GPU_OK))
    with pkg.Aligner(0, 4 << 30) as al:
        alone = []
        for b, pen, kw, code in plan:
            if b is nooff:
                alone.append(al.align(packed, pen))
            elif code == pkg.WFA_GPU_OK:
                alone.append(al.align(b, pen, score_only=kw.get("score_only", False)))
            elif code == pkg.WFA_GPU_ECIGAR_CAPACITY:
                alone.append(al.align(b, pen))
            else:
                alone.append(None)
    with pkg.Server(0, workers=1, memory_budget_bytes=16 << 30) as srv:
        ids = [srv.submit(b, pen, **kw) for b, pen, kw, _ in plan]
        outs = [srv.wait(i, check=False) for i in ids]
    for (b, pen, kw, code), (got, st), want in zip(plan, outs, alone):
        assert st.result == code, (st.result, code)
        if want is None:
            continue
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
        if kw.get("score_only"):
            continue
        assert np.array_equal(got[3], want[3])  # offsets, also when the capacity was short
        if code == pkg.WFA_GPU_OK:
            assert np.array_equal(got[2], want[2])


def test_large_need_waits_while_small_ones_run(pkg, oracle_mod):
    """A request whose estimated wavefront need does not fit the free arena
    waits while requests queued after it, with small needs, pass it and
    run.  Arena of 192 MiB: small calls take 64 MiB slices; the large request
    (60 pairs of 5 kbp: above 1 GiB at the 10% edit-rate bound) a slice of
    half the arena, 96 MiB, which the first two small calls leave no room
    for.  Every result equals the request aligned alone."""
    from paper_2204_02085_gb300 import synth

    small = [synth.uniform_reads(3000, 100, 3, seed=600 + j) for j in range(5)]
    big = synth.long_reads(60, 5000, 0.01, 0.02, seed=610)
    # distinct max_score values keep the first two small requests and the
    # large one in calls of their own (merging joins only equal parameters)
    bounds = [0, 100000, 0, 0, 0]
    with pkg.Aligner(0, 2 << 30) as al:
        alone_small = [al.align(b, (4, 6, 2), max_score=ms) for b, ms in zip(small, bounds)]
        alone_big = al.align(big, (4, 6, 2), max_score=1 << 20)
    with pkg.Server(0, workers=4, memory_budget_bytes=192 << 20) as srv:
        ids = [srv.submit(small[j], (4, 6, 2), max_score=bounds[j], cigar_capacity=_cap(small[j])) for j in (0, 1)]
        big_id = srv.submit(big, (4, 6, 2), max_score=1 << 20, cigar_capacity=_cap(big))
        ids += [srv.submit(small[j], (4, 6, 2), max_score=bounds[j], cigar_capacity=_cap(small[j]))
                for j in (2, 3, 4)]
        outs = [srv.wait(i) for i in ids]
        big_out, big_st = srv.wait(big_id)
    stats = [st for _, st in outs]
    assert big_st.result == pkg.WFA_GPU_OK and all(st.result == pkg.WFA_GPU_OK for st in stats)
    # requests submitted after the large one started before it
    assert any(st.start_s < big_st.start_s for st in stats[2:])
    for (got, _), want in zip(outs, alone_small):
        for x, y in zip(got, want):
            assert np.array_equal(x, y)
    for x, y in zip(big_out, alone_big):
        assert np.array_equal(x, y)
    o = oracle_mod.wfa_batch(big, (4, 6, 2), nthreads=16)
    assert np.array_equal(big_out[0], o[0]) and np.array_equal(big_out[2], o[2])
