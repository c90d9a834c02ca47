"""The seeded input generator: deterministic, the paper's workload shape."""

import numpy as np

from paper_2204_02085_gb300 import synth


def _lev(a, b):
    prev = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        cur = [i] + [0] * len(b)
        for j in range(1, len(b) + 1):
            cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + (a[i - 1] != b[j - 1]))
        prev = cur
    return prev[-1]


def test_deterministic_and_shaped():
    a = synth.uniform_reads(3000, 100, 2, seed=0)
    b = synth.uniform_reads(3000, 100, 2, seed=0)
    c = synth.uniform_reads(3000, 100, 2, seed=1)
    assert a.sha256() == b.sha256() != c.sha256()
    assert a.n == 3000
    assert np.all(a.text_lengths == 100)
    assert set(np.unique(a.pattern_lengths)) <= {98, 99, 100, 101, 102}
    assert set(np.unique(a.patterns)) <= set(b"ACGT") and set(np.unique(a.texts)) <= set(b"ACGT")
    assert a.patterns.size == a.pattern_lengths.sum() and a.texts.size == a.text_lengths.sum()
    assert a.pattern_offsets[0] == 0 and np.all(np.diff(a.pattern_offsets) == a.pattern_lengths[:-1])


def test_edit_distance_at_most_edits():
    """Each pattern is the text after k edits: unit edit distance <= k, and
    for most pairs exactly k (edits rarely cancel)."""
    for k in (2, 4):
        b = synth.uniform_reads(200, 100, k, seed=5)
        d = np.array([_lev(*b.pair(i)) for i in range(b.n)])
        assert d.max() <= k
        assert np.mean(d == k) > 0.8


def test_chunking_is_invisible_to_callers():
    """A batch that spans several generator chunks is the same function of
    its arguments every time, and its first pairs are those of a smaller
    batch drawn with the same seed only within the first chunk."""
    n = synth.CHUNK + 17
    a = synth.uniform_reads(n, 20, 1, seed=3)
    b = synth.uniform_reads(n, 20, 1, seed=3)
    assert a.sha256() == b.sha256() and a.n == n


def test_from_pairs_and_subset():
    pairs = [(b"ACG", b"AC"), (b"", b"T"), (b"acgt", b"")]
    b = synth.from_pairs(pairs)
    assert [b.pair(i) for i in range(3)] == pairs
    s = b.subset([2, 0])
    assert [s.pair(i) for i in range(2)] == [pairs[2], pairs[0]]


def test_reads_in_windows_shape_and_determinism():
    from paper_2204_02085_gb300 import synth

    a = synth.reads_in_windows(300, 100, 50, 3, seed=11)
    b = synth.reads_in_windows(300, 100, 50, 3, seed=11)
    assert a.sha256() == b.sha256()
    core = synth.uniform_reads(300, 100, 3, seed=11)
    for i in range(a.n):
        read, window = a.pair(i)
        edited, original = core.pair(i)
        assert read == original and len(read) == 100
        assert edited in window and len(edited) <= len(window) <= len(edited) + 100
