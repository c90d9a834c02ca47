"""The lane-per-pair short-read kernel (one lane per pair, the warp's 32
pairs in lockstep) against the oracle, bit for bit: every store size forced
in turn, six penalty sets, ragged lengths 0..127, unrelated pairs, score
bounds and score-only calls; and the shared-lane kernel it replaced, which
still runs when the lane variants are turned off (WFA_GPU_LANE=0)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LANE_NAMES = ("lane_l127_c40", "lane_l127_c64", "lane_l127_c104", "lane_l127_c197")
# the geometry of scaled penalties x = 2, o + e = 4, e = 1 compiled in
CT_NAMES = ("lane_ct241_l127_c40", "lane_ct241_l127_c64", "lane_ct241_l127_c104", "lane_ct241_l127_c197")


@pytest.fixture(scope="module")
def pkg():
    from paper_2204_02085_gb300 import build

    build.build()
    import paper_2204_02085_gb300 as p

    return p


def _variant_index(pkg, name):
    with pkg.Aligner(0, 1 << 28) as al:
        for i in range(64):
            nm = al.variant_name(i)
            if nm is None:
                break
            if nm == name:
                return i
    raise AssertionError("variant %s not in the plan" % name)


def _batch(seed):
    """100 bp reads at 0-8 edits, ragged lengths 0-127 and unrelated pairs."""
    from paper_2204_02085_gb300 import synth

    rng = np.random.default_rng(seed)
    parts = [synth.uniform_reads(400, 100, e, seed=seed + e) for e in (0, 1, 2, 3, 4, 6, 8)]
    pairs = [p.pair(i) for p in parts for i in range(p.n)]
    for _ in range(300):
        n, m = int(rng.integers(0, 128)), int(rng.integers(0, 128))
        a = bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, n)])
        if rng.random() < 0.5:
            b = bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, m)])
        else:  # a related text: a's prefix with a few substitutions
            b = bytearray(a[:m] + bytes(np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, max(0, m - n))]))
            for j in rng.integers(0, max(1, len(b)), 3):
                if len(b):
                    b[int(j) % len(b)] = b"ACGT"[int(rng.integers(0, 4))]
            b = bytes(b)
        pairs.append((a, b))
    pairs += [(b"", b""), (b"A", b""), (b"", b"C"), (b"AAAA", b"AAA"), (b"A" * 127, b"A" * 127),
              (b"A" * 127, b"C" * 127), (b"acgt" * 31, b"ACGT" * 31 + b"AC")]
    return synth.from_pairs(pairs)


def _check(got, want):
    s, st, w, off = got
    ws, wst, ww, woff = want
    assert np.array_equal(st, wst), "status differs"
    assert np.array_equal(s, ws), "scores differ"
    assert np.array_equal(off, woff), "CIGAR offsets differ"
    assert np.array_equal(w, ww), "CIGAR words differ"


@pytest.mark.parametrize("name", LANE_NAMES)
@pytest.mark.parametrize("pen", [(4, 6, 2), (2, 3, 1), (5, 1, 3), (3, 2, 2), (16, 6, 2), (6, 4, 2)])
def test_each_store_matches_oracle(pkg, oracle_mod, monkeypatch, name, pen):
    vi = _variant_index(pkg, name)
    monkeypatch.setenv("WFA_GPU_SHORT_VARIANT", str(vi))
    batch = _batch(500 + vi)
    want = oracle_mod.wfa_batch(batch, pen, nthreads=8)
    with pkg.Aligner(0, 1 << 30) as al:
        got = al.align(batch, pen)
        assert al.variant_name(al.timing()["short_variant"]) == name
        _check(got, want)
        so = al.align(batch, pen, score_only=True)
        assert np.array_equal(so[0], want[0]) and np.array_equal(so[1], want[1])


@pytest.mark.parametrize("name", CT_NAMES)
@pytest.mark.parametrize("pen", [(4, 6, 2), (2, 3, 1), (8, 12, 4)])
def test_compiled_geometry_matches_oracle(pkg, oracle_mod, monkeypatch, name, pen):
    """Penalty sets that scale to 2/4/1 run the compiled-geometry variants."""
    vi = _variant_index(pkg, name)
    monkeypatch.setenv("WFA_GPU_SHORT_VARIANT", str(vi))
    batch = _batch(700 + vi)
    want = oracle_mod.wfa_batch(batch, pen, nthreads=8)
    with pkg.Aligner(0, 1 << 30) as al:
        got = al.align(batch, pen)
        assert al.variant_name(al.timing()["short_variant"]) == name
        _check(got, want)
        so = al.align(batch, pen, score_only=True)
        assert np.array_equal(so[0], want[0]) and np.array_equal(so[1], want[1])


def test_compiled_geometry_only_for_its_penalties(pkg, oracle_mod, monkeypatch):
    """Forcing a compiled-geometry variant on other penalties is ignored."""
    monkeypatch.setenv("WFA_GPU_SHORT_VARIANT", str(_variant_index(pkg, CT_NAMES[3])))
    batch = _batch(777)
    for pen in ((5, 1, 3), (6, 4, 2)):
        want = oracle_mod.wfa_batch(batch, pen, nthreads=8)
        with pkg.Aligner(0, 1 << 30) as al:
            got = al.align(batch, pen)
            assert not al.variant_name(al.timing()["short_variant"]).startswith("lane_ct")
            _check(got, want)


@pytest.mark.parametrize("name", ("lane_l127_c40", "lane_l127_c197", "lane_ct241_l127_c40", "lane_ct241_l127_c197"))
def test_score_bounds(pkg, oracle_mod, monkeypatch, name):
    """max_score at, below and above the stored scores: SCORE_LIMIT beyond the
    bound, deferral to the arena kernels beyond the store."""
    vi = _variant_index(pkg, name)
    monkeypatch.setenv("WFA_GPU_SHORT_VARIANT", str(vi))
    batch = _batch(900)
    with pkg.Aligner(0, 1 << 30) as al:
        for bound in (1, 8, 14, 16, 17, 30, 33, 64):
            want = oracle_mod.wfa_batch(batch, (4, 6, 2), max_score=bound, nthreads=8)
            _check(al.align(batch, (4, 6, 2), max_score=bound), want)


def test_paper_batches_every_store(pkg, oracle_mod, monkeypatch):
    """50,000 pairs of the paper's 100 bp workload at 2 and 4 edits through
    each store: pairs past a small store go to the arena kernels, the
    results stay the same."""
    from paper_2204_02085_gb300 import synth

    for e in (2, 4):
        batch = synth.uniform_reads(50_000, 100, e, seed=40 + e)
        want = oracle_mod.wfa_batch(batch, (4, 6, 2), nthreads=16)
        for name in LANE_NAMES + CT_NAMES:
            monkeypatch.setenv("WFA_GPU_SHORT_VARIANT", str(_variant_index(pkg, name)))
            with pkg.Aligner(0, 1 << 30) as al:
                _check(al.align(batch, (4, 6, 2)), want)


def test_autotuner_picks_a_lane_store(pkg, oracle_mod):
    from paper_2204_02085_gb300 import synth

    for e, expect in ((2, "lane_ct241_l127_c40"), (4, "lane_l127_c197")):
        batch = synth.uniform_reads(20_000, 100, e, seed=60 + e)
        with pkg.Aligner(0, 1 << 30) as al:
            got = al.align(batch, (4, 6, 2))
            assert al.variant_name(al.timing()["short_variant"]) == expect
        _check(got, oracle_mod.wfa_batch(batch, (4, 6, 2), nthreads=16))


def test_shared_lane_kernel_still_matches(pkg, oracle_mod, monkeypatch):
    """WFA_GPU_LANE=0: the shared-lane kernel runs the short pairs."""
    monkeypatch.setenv("WFA_GPU_LANE", "0")
    batch = _batch(1234)
    want = oracle_mod.wfa_batch(batch, (4, 6, 2), nthreads=8)
    with pkg.Aligner(0, 1 << 30) as al:
        got = al.align(batch, (4, 6, 2))
        assert not al.variant_name(al.timing()["short_variant"]).startswith("lane")
        _check(got, want)


@pytest.mark.parametrize("order", ["0", "1"])
@pytest.mark.parametrize("name", ("lane_l127_c40", "lane_l127_c197", "lane_ct241_l127_c104"))
def test_input_order_does_not_change_results(pkg, oracle_mod, monkeypatch, order, name):
    """The lane kernel's pairs sorted by estimated score in groups
    (default) or taken in call order: the same results, bit for bit, on a
    batch whose size is no multiple of the group and that holds pairs
    longer than the kernel takes, pairs with other bytes than A/C/G/T and
    empty sequences."""
    from paper_2204_02085_gb300 import synth

    monkeypatch.setenv("WFA_GPU_LANE_ORDER", order)
    monkeypatch.setenv("WFA_GPU_SHORT_VARIANT", str(_variant_index(pkg, name)))
    base = _batch(4242)
    pairs = [base.pair(i) for i in range(base.n)]
    rng = np.random.default_rng(17)
    extra = [(b"ACGT" * 40, b"ACGA" * 40), (b"ACGNT", b"ACGT"), (b"", b""), (b"ACGT", b"AC-T"),
             (b"A" * 128, b"A" * 127), (b"C" * 127, b"C" * 128)]
    for pr in extra:
        pairs.insert(int(rng.integers(0, 1500)), pr)
    pairs = pairs[:2 * 1024 + 77]  # two groups of 1,024 and a ragged third
    batch = synth.from_pairs(pairs)
    pen = (4, 6, 2)
    want = oracle_mod.wfa_batch(batch, pen, nthreads=8)
    with pkg.Aligner(0, 1 << 30) as al:
        _check(al.align(batch, pen), want)
        for bound in (8, 16):
            _check(al.align(batch, pen, max_score=bound), oracle_mod.wfa_batch(batch, pen, max_score=bound, nthreads=8))
        so = al.align(batch, pen, score_only=True)
        assert np.array_equal(so[0], want[0]) and np.array_equal(so[1], want[1])


@pytest.mark.parametrize("e", (2, 4))
def test_ordered_paper_batch_launch_count(pkg, oracle_mod, monkeypatch, e):
    """Default path on the paper's workload: the ordering pass runs (one more
    launch than in call order, for the autotuner's sample run and for the
    main run) and the results match the oracle."""
    from paper_2204_02085_gb300 import synth

    batch = synth.uniform_reads(100_003, 100, e, seed=80 + e)
    want = oracle_mod.wfa_batch(batch, (4, 6, 2), nthreads=16)
    launches = {}
    for order in ("0", "1"):
        monkeypatch.setenv("WFA_GPU_LANE_ORDER", order)
        with pkg.Aligner(0, 1 << 30) as al:
            _check(al.align(batch, (4, 6, 2)), want)
            launches[order] = al.timing()["kernel_launches"]
    assert launches["1"] == launches["0"] + 2


@pytest.mark.parametrize("sort_min", ["0", "99"])
@pytest.mark.parametrize("name", ("lane_ct241_l127_c40", "lane_l127_c197"))
def test_sorted_and_pack_only_ordering_agree(pkg, oracle_mod, monkeypatch, sort_min, name):
    """The ordering pass sorting every store's groups (WFA_GPU_LANE_SORT_MIN=0)
    or packing them in call order (99): the oracle's results either way."""
    from paper_2204_02085_gb300 import synth

    monkeypatch.setenv("WFA_GPU_LANE_SORT_MIN", sort_min)
    monkeypatch.setenv("WFA_GPU_SHORT_VARIANT", str(_variant_index(pkg, name)))
    batch = synth.uniform_reads(30_001, 100, 4, seed=91)
    want = oracle_mod.wfa_batch(batch, (4, 6, 2), nthreads=16)
    with pkg.Aligner(0, 1 << 30) as al:
        _check(al.align(batch, (4, 6, 2)), want)


@pytest.mark.parametrize("n", [1, 31, 33, 1023, 1024, 1025, 2048])
@pytest.mark.parametrize("name", ("lane_ct241_l127_c40", "lane_l127_c197"))
def test_ordering_partial_groups(pkg, oracle_mod, monkeypatch, n, name):
    """Batches of one pair, part of a warp, part of a group, whole groups and
    just past a group, through the packing-only (40-cell store) and the
    sorting (197-cell store) ordering: the oracle's results."""
    from paper_2204_02085_gb300 import synth

    monkeypatch.setenv("WFA_GPU_SHORT_VARIANT", str(_variant_index(pkg, name)))
    batch = synth.uniform_reads(n, 100, 4, seed=1000 + n)
    want = oracle_mod.wfa_batch(batch, (4, 6, 2), nthreads=8)
    with pkg.Aligner(0, 1 << 30) as al:
        _check(al.align(batch, (4, 6, 2)), want)
        assert al.timing()["kernel_launches"] > 0
