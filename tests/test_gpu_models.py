"""Penalty models beside gap-affine: the gap-linear model (o = 0, every gap
column costs e) and its unit-cost case, the edit distance (x = e = 1).  The
short kernel stores only the M wavefronts for them (I and D follow from M
when o = 0) and must give bit-exactly the scores, status and canonical
CIGARs of the oracle run with the same penalties."""

import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
NCPU = os.cpu_count() or 4
LINEAR_SETS = [(1, 0, 1), (3, 0, 2), (2, 0, 3), (5, 0, 1)]


@pytest.fixture(scope="module")
def pkg():
    from paper_2204_02085_gb300 import build

    build.build()
    import paper_2204_02085_gb300 as p

    return p


@pytest.fixture(scope="module")
def al(pkg):
    a = pkg.Aligner(0, 2 << 30)
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


def run(al, oracle, b, pen, max_score=0, score_only=False):
    got = al.align(b, pen, max_score=max_score, score_only=score_only, timing=True)
    want = oracle.wfa_batch(b, pen, max_score=max_score, want_cigar=not score_only, nthreads=NCPU)
    same(got, want, score_only)
    return al.timing()


@pytest.mark.parametrize("pen", LINEAR_SETS)
@pytest.mark.parametrize("edits", [2, 4, 8])
def test_linear_100bp(al, oracle_mod, pen, edits):
    """100 bp reads (the paper's shape) under gap-linear penalties: the
    M-only short-kernel variants run them."""
    from paper_2204_02085_gb300 import synth

    b = synth.uniform_reads(60_000, 100, edits, seed=70 + edits)
    t = run(al, oracle_mod, b, pen)
    assert t["short_variant"] >= 0
    assert al.variant_name(t["short_variant"]).endswith("lin"), al.variant_name(t["short_variant"])
    if edits <= 4:
        # the M-only store holds these scores: the short kernel itself
        # finishes (nearly) every pair
        assert t["deferred_pairs"] <= b.n // 100, t["deferred_pairs"]


@pytest.mark.parametrize("pen", LINEAR_SETS)
def test_linear_ragged_unrelated_and_bounds(al, oracle_mod, pen):
    """Lengths 0..255 (int8 and int16 variants, deferrals to the arena),
    unrelated pairs (high scores), score bounds, score-only."""
    from paper_2204_02085_gb300 import synth

    rag = synth.random_pairs(3000, 0, 255, seed=81, edit_rate=0.05)
    unr = synth.random_pairs(300, 0, 300, seed=82)
    b = synth.from_pairs([rag.pair(i) for i in range(rag.n)] + [unr.pair(i) for i in range(unr.n)])
    run(al, oracle_mod, b, pen)
    run(al, oracle_mod, b, pen, score_only=True)
    for ms in (3, 17, 60):
        run(al, oracle_mod, b, pen, max_score=ms)
    # the short pairs alone, each bound inside the store: the short kernel
    # decides every pair (no deferral)
    short = b.subset(np.nonzero((b.pattern_lengths <= 127) & (b.text_lengths <= 127))[0])
    for ms in (1, 3, 6):
        t = run(al, oracle_mod, short, pen, max_score=ms)
        assert t["deferred_pairs"] == 0, t


def test_edit_distance_is_levenshtein(al, oracle_mod):
    """x = e = 1, o = 0: every score equals the textbook unit-cost edit
    distance (computed here independently of the oracle)."""
    from paper_2204_02085_gb300 import synth

    def lev(a, b):
        prev = list(range(len(b) + 1))
        for i in range(1, len(a) + 1):
            cur = [i] + [0] * len(b)
            for j in range(1, len(b) + 1):
                cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + (a[i - 1] != b[j - 1]))
            prev = cur
        return prev[-1]

    b = synth.uniform_reads(300, 100, 6, seed=90)
    s, st, _, _ = al.align(b, (1, 0, 1))
    for i in range(b.n):
        p, t = b.pair(i)
        assert st[i] == 0 and s[i] == lev(p, t)
