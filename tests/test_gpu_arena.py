"""Parity of the arena path (pairs the short-read kernel defers: medium and
long reads, high scores) with the CPU oracle, bit-exact, through the C ABI.

Workloads: the long-read configuration (10 kbp pairs, edit rate 1-5 %,
seed 4) on a subset, the mixed-length configuration (100-2,000 bp,
edit rate 0-10 %, tandem repeats, seed 3) on a subset, unrelated pairs (high
scores), score-only (ring storage) and retries through a small arena.
"""

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


def same(got, want, score_only=False):
    s, st, w, off = got
    os_, ost, ow, ooff = want
    bad = np.nonzero((s != os_) | (st != ost))[0]
    assert bad.size == 0, "pairs %s: gpu %s/%s oracle %s/%s" % (bad[:5], s[bad[:5]], st[bad[:5]], os_[bad[:5]],
                                                               ost[bad[:5]])
    if not score_only:
        assert np.array_equal(off, ooff), "CIGAR offsets differ"
        assert np.array_equal(w, ow), "CIGAR words differ"


def both_modes(pkg, oracle, batch, pen=(4, 6, 2), scratch=0, max_score=0):
    want = oracle.wfa_batch(batch, pen, max_score=max_score, nthreads=NCPU)
    with pkg.Aligner(0, scratch_bytes=scratch) as al:
        got = al.align(batch, pen, max_score=max_score)
        same(got, want)
        got_so = al.align(batch, pen, max_score=max_score, score_only=True)
        same(got_so, want, score_only=True)
        return al.timing()


def test_long_reads_subset(pkg, oracle_mod):
    """First 60 pairs of the long-read configuration (10 kbp, 1-5 %)."""
    from paper_2204_02085_gb300 import synth

    b = synth.long_reads(60, 10_000, 0.01, 0.05, seed=4)
    t = both_modes(pkg, oracle_mod, b, scratch=8 << 30)
    assert t["deferred_pairs"] == b.n  # every pair took the one-CTA arena kernel


def test_long_reads_retry_small_arena(pkg, oracle_mod):
    """An arena too small for the first pass: pairs are retried with fewer,
    larger slices and still match."""
    from paper_2204_02085_gb300 import synth

    b = synth.long_reads(12, 10_000, 0.03, 0.05, seed=40)
    both_modes(pkg, oracle_mod, b, scratch=256 << 20)


def test_mixed_lengths_subset(pkg, oracle_mod):
    """First 4,000 pairs of the mixed-length configuration."""
    from paper_2204_02085_gb300 import synth

    b = synth.mixed_reads(4000, seed=3)
    both_modes(pkg, oracle_mod, b, scratch=4 << 30)


@pytest.mark.parametrize("pen", [(4, 6, 2), (1, 0, 1), (16, 6, 2), (2, 3, 1)])
def test_unrelated_medium_and_long(pkg, oracle_mod, pen):
    from paper_2204_02085_gb300 import synth

    med = synth.random_pairs(40, 200, 2048, seed=61)
    lng = synth.random_pairs(3, 2049, 4000, seed=62)
    b = synth.from_pairs([med.pair(i) for i in range(med.n)] + [lng.pair(i) for i in range(lng.n)])
    both_modes(pkg, oracle_mod, b, pen=pen, scratch=4 << 30)


def test_score_bound_on_arena_pairs(pkg, oracle_mod):
    from paper_2204_02085_gb300 import synth

    b = synth.mixed_reads(800, seed=33)
    for ms in (40, 200, 1000):
        both_modes(pkg, oracle_mod, b, scratch=2 << 30, max_score=ms)


def test_long_reads_config_parity_500(pkg, oracle_mod):
    """The long-read configuration's first 500 pairs (20,000-pair workload,
    seed 4), bit-exact, score + CIGAR and score only."""
    from paper_2204_02085_gb300 import synth

    b = synth.long_reads(500, 10_000, 0.01, 0.05, seed=4)
    both_modes(pkg, oracle_mod, b, scratch=32 << 30)
