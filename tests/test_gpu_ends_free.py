"""Ends-free alignment on the GPU (wfa_gpu_set_ends_free): free leading and
trailing pattern / text characters, bit-exact against the oracle run with
the same free lengths -- scores, status, canonical CIGARs (including the
skipped ends as D / I runs) -- on the short kernel and both arena team
sizes, with score bounds, score-only calls and graph replays."""

import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 4


@pytest.fixture(scope="module")
def pkg():
    from paper_2204_02085_gb300 import build

    build.build()
    import paper_2204_02085_gb300 as p

    return p


@pytest.fixture()
def al(pkg):
    a = pkg.Aligner(0, 4 << 30)
    yield a
    a.close()


def same(got, want, score_only=False):
    s, st, w, off = got
    os_, ost, ow, ooff = want
    bad = np.nonzero((s != os_) | (st != ost))[0]
    assert bad.size == 0, "pairs %s: gpu %s/%s oracle %s/%s" % (bad[:5], s[bad[:5]], st[bad[:5]], os_[bad[:5]],
                                                               ost[bad[:5]])
    if not score_only:
        assert np.array_equal(off, ooff), "CIGAR offsets differ"
        assert np.array_equal(w, ow), "CIGAR words differ"


def run(al, oracle, b, pen, ends, max_score=0, score_only=False):
    al.set_ends_free(*ends)
    got = al.align(b, pen, max_score=max_score, score_only=score_only, timing=True)
    want = oracle.wfa_batch(b, pen, max_score=max_score, want_cigar=not score_only, nthreads=NCPU, ends=ends)
    same(got, want, score_only)
    return al.timing()


def embedded(n_pairs, plen, flank, edits, seed):
    """Patterns of plen bases; each text = random left flank + the pattern
    after `edits` edits + random right flank (flanks 0..flank bases)."""
    from paper_2204_02085_gb300 import synth

    rng = np.random.Generator(np.random.PCG64(seed))
    core = synth.uniform_reads(n_pairs, plen, edits, seed=seed)
    pairs = []
    for i in range(n_pairs):
        p, t = core.pair(i)  # pattern = edited text; use the text as the read
        lf = bytes(b"ACGT"[j] for j in rng.integers(0, 4, size=int(rng.integers(0, flank + 1))))
        rf = bytes(b"ACGT"[j] for j in rng.integers(0, 4, size=int(rng.integers(0, flank + 1))))
        pairs.append((t, lf + p + rf))
    return synth.from_pairs(pairs)


@pytest.mark.parametrize("ends", [(3, 3, 3, 3), (0, 0, 6, 6), (6, 6, 0, 0), (2, 0, 0, 5), (0, 4, 4, 0)])
@pytest.mark.parametrize("edits", [2, 4])
def test_short_reads_small_free_ends(al, oracle_mod, ends, edits):
    from paper_2204_02085_gb300 import synth

    b = synth.uniform_reads(40_000, 100, edits, seed=100 + edits)
    t = run(al, oracle_mod, b, (4, 6, 2), ends)
    assert t["short_variant"] >= 0


@pytest.mark.parametrize("pen", [(4, 6, 2), (1, 0, 1), (3, 0, 2), (2, 3, 1)])
def test_semi_global_read_in_reference_window(al, oracle_mod, pen):
    """A read aligned to its best-matching stretch of a longer text: text
    ends free over the whole text (medium lengths: arena one-warp teams)."""
    b = embedded(1500, 100, 120, 3, seed=7)
    m = int(b.text_lengths.max())
    run(al, oracle_mod, b, pen, (0, 0, m, m))


def test_semi_global_long(al, oracle_mod):
    """Long texts (one-CTA teams): 2,200-3,000 bp windows around a read."""
    b = embedded(60, 2200, 400, 60, seed=8)
    m = int(b.text_lengths.max())
    run(al, oracle_mod, b, (4, 6, 2), (0, 0, m, m))
    run(al, oracle_mod, b, (4, 6, 2), (0, 0, m, m), score_only=True)


def test_ragged_random_ends_bounds_and_score_only(al, oracle_mod):
    from paper_2204_02085_gb300 import synth

    rng = np.random.default_rng(9)
    rag = synth.random_pairs(3000, 0, 255, seed=91, edit_rate=0.05)
    for pen in [(4, 6, 2), (3, 0, 2)]:
        for _ in range(3):
            ends = tuple(int(v) for v in rng.integers(0, 40, size=4))
            run(al, oracle_mod, rag, pen, ends)
            run(al, oracle_mod, rag, pen, ends, score_only=True)
            run(al, oracle_mod, rag, pen, ends, max_score=20)


def test_everything_free_scores_zero(al, oracle_mod):
    from paper_2204_02085_gb300 import synth

    b = synth.random_pairs(2000, 0, 200, seed=93)
    t = run(al, oracle_mod, b, (4, 6, 2), (255, 255, 255, 255))
    s, st, _, _ = al.align(b, (4, 6, 2))
    assert (s == 0).all() and (st == 0).all()
    assert t["deferred_pairs"] >= 0


def test_graph_replay_and_switch(pkg, oracle_mod):
    """Graph mode keys on the free lengths: a replay with the same lengths
    reproduces the eager result, other lengths capture a new graph."""
    import torch

    from paper_2204_02085_gb300 import synth

    b = synth.uniform_reads(20_000, 100, 3, seed=94)
    dev = torch.device("cuda:0")
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)  # noqa: E731
    pat, plen, txt, tlen = t(b.patterns), t(b.pattern_lengths), t(b.texts), t(b.text_lengths)
    n = b.n
    s = torch.empty(n, dtype=torch.int32, device=dev)
    st = torch.empty(n, dtype=torch.int8, device=dev)
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    w = torch.empty(24 * n, dtype=torch.int32, device=dev)
    with pkg.Aligner(0) as al:
        for ends in [(4, 4, 4, 4), (0, 0, 0, 0), (4, 4, 4, 4), (0, 9, 9, 0)]:
            al.set_ends_free(*ends)
            for _ in range(2):
                assert al.align_device(pat, None, plen, txt, None, tlen, s, st, w, off, graph=True) == 0
                torch.cuda.synchronize()
                want = oracle_mod.wfa_batch(b, (4, 6, 2), nthreads=NCPU, ends=ends)
                o = off.cpu().numpy()
                got = (s.cpu().numpy(), st.cpu().numpy(), w.cpu().numpy()[: int(o[-1])].view(np.uint32), o)
                same(got, want)


def test_setter_rejects_bad_lengths(pkg):
    with pkg.Aligner(0) as al:
        with pytest.raises(pkg.WfaGpuError):
            al.set_ends_free(-1, 0, 0, 0)
        al.set_ends_free(0, 0, 0, 0)
