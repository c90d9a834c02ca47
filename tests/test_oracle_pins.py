"""Pins for the CPU oracle, against things other than itself.

The oracle computes the minimum-cost gap-affine global alignment (the result
the wavefront algorithm, WFA, reaches exactly; the paper runs it unmodified,
Sec. I) and a canonical alignment under a fixed tie-break.  Each check below
compares it with an independent source:

* brute-force enumeration of every alignment (exhaustive for lengths <= 4,
  random for lengths <= 6) -- the definition itself;
* special cases that reduce to textbook routines written here in Python:
  Levenshtein distance for (x, o, e) = (1, 0, 1), LCS for o = 0, x > 2e;
* closed forms: identical strings, one substitution, one gap of length k;
* invariants: score symmetry under swapping pattern/text, every alignment
  rescores to its score and consumes both sequences;
* hand-derived golden cases (tests/golden/tie_break_cases.txt).
"""

import itertools
import random

import numpy as np
import pytest

# gap-affine sets, and gap-linear ones (o = 0: every gap column costs e; the
# edit distance at x = e = 1)
PENALTY_SETS = [(4, 6, 2), (1, 0, 1), (2, 3, 1), (5, 1, 3), (3, 2, 2), (16, 6, 2), (3, 0, 2), (2, 0, 3)]


def all_seqs(max_len):
    return ["".join(p) for L in range(max_len + 1) for p in itertools.product("ACGT", repeat=L)]


def swap_id(ops):
    return ops.translate(str.maketrans("ID", "DI"))


def levenshtein(a, b):
    """Textbook unit-cost edit distance."""
    prev = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        cur = [i] + [0] * len(b)
        for j in range(1, len(b) + 1):
            cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + (a[i - 1] != b[j - 1]))
        prev = cur
    return prev[-1]


def lcs(a, b):
    """Textbook longest-common-subsequence length."""
    prev = [0] * (len(b) + 1)
    for i in range(1, len(a) + 1):
        cur = [0] * (len(b) + 1)
        for j in range(1, len(b) + 1):
            cur[j] = prev[j - 1] + 1 if a[i - 1] == b[j - 1] else max(prev[j], cur[j - 1])
        prev = cur
    return prev[-1]


def check_pair(oracle, p, t, pen):
    bs, bops, _ = oracle.brute(p, t, pen)
    gs, gops = oracle.gotoh(p, t, pen)
    st, ws, wops = oracle.wfa(p, t, pen)
    assert st == oracle.OK
    assert bs == gs == ws, (p, t, pen, bs, gs, ws)
    assert oracle.rescore(p, t, wops, pen) == ws
    assert wops == gops == bops, (p, t, pen, bops, gops, wops)


@pytest.mark.parametrize("pen", [(4, 6, 2), (1, 0, 1), (16, 6, 2), (3, 0, 2)])
def test_exhaustive_lengths_upto_4(oracle_mod, pen):
    """Every pair of A/C/G/T strings of length <= 4 (341^2 pairs): brute
    force, Gotoh and WFA agree on the score and on the canonical alignment."""
    seqs = all_seqs(4)
    for p in seqs:
        for t in seqs:
            check_pair(oracle_mod, p, t, pen)


@pytest.mark.parametrize("pen", PENALTY_SETS)
def test_random_lengths_upto_6(oracle_mod, pen):
    rng = random.Random(hash(pen) & 0xFFFF)
    for _ in range(1500):
        p = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 6)))
        t = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 6)))
        check_pair(oracle_mod, p, t, pen)


def test_small_alphabet_ties(oracle_mod):
    """Two-letter strings make ties (repeats) common: the tie-break of the
    three implementations must still agree with brute force."""
    rng = random.Random(7)
    for pen in PENALTY_SETS:
        for _ in range(600):
            p = "".join(rng.choice("AC") for _ in range(rng.randint(0, 6)))
            t = "".join(rng.choice("AC") for _ in range(rng.randint(0, 6)))
            check_pair(oracle_mod, p, t, pen)


def test_levenshtein_special_case(oracle_mod):
    """(x, o, e) = (1, 0, 1): every column costs 1, so the score is the unit
    edit distance."""
    rng = random.Random(11)
    for _ in range(400):
        p = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 30)))
        t = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 30)))
        d = levenshtein(p, t)
        assert oracle_mod.gotoh(p, t, (1, 0, 1), want_ops=False)[0] == d
        st, s, ops = oracle_mod.wfa(p, t, (1, 0, 1))
        assert s == d and oracle_mod.rescore(p, t, ops, (1, 0, 1)) == d


@pytest.mark.parametrize("pen", [(5, 0, 2), (3, 0, 1), (7, 0, 3)])
def test_lcs_special_case(oracle_mod, pen):
    """o = 0 and x > 2e: a mismatch never pays, each unmatched character costs
    e, so the score is e * (n + m - 2 LCS)."""
    x, o, e = pen
    rng = random.Random(x * 100 + e)
    for _ in range(300):
        p = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 25)))
        t = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 25)))
        want = e * (len(p) + len(t) - 2 * lcs(p, t))
        assert oracle_mod.gotoh(p, t, pen, want_ops=False)[0] == want
        assert oracle_mod.wfa(p, t, pen)[1] == want


@pytest.mark.parametrize("pen", PENALTY_SETS)
def test_closed_forms(oracle_mod, pen):
    x, o, e = pen
    rng = random.Random(3)
    for _ in range(100):
        n = rng.randint(1, 60)
        s = "".join(rng.choice("ACGT") for _ in range(n))
        # identical strings: 0 and nM
        st, sc, ops = oracle_mod.wfa(s, s, pen)
        assert (sc, ops) == (0, "M" * n)
        # one substitution: x when x <= 2(o+e) (else two gaps are cheaper);
        # the alignment is aM1XbM when x < 2(o+e).  At x == 2(o+e) an I/D pair
        # ties with the X and may lie further right, which the canonical rule
        # prefers, so only the score is fixed there.
        i = rng.randrange(n)
        sub = s[:i] + rng.choice([c for c in "ACGT" if c != s[i]]) + s[i + 1:]
        st, sc, ops = oracle_mod.wfa(sub, s, pen)
        if x <= 2 * (o + e):
            assert sc == x
            if x < 2 * (o + e):
                assert ops == "M" * i + "X" + "M" * (n - i - 1)
        else:
            assert sc == 2 * (o + e)
        assert oracle_mod.gotoh(sub, s, pen, want_ops=False)[0] == sc
        # one gap of length k: exactly o + k e in any context (at least k gap
        # columns of one kind are needed, and one run achieves it)
        k = rng.randint(1, min(8, n))
        j = rng.randint(0, n - k)
        dele = s[:j] + s[j + k:]
        assert oracle_mod.wfa(s, dele, pen)[1] == o + k * e  # pattern longer: D
        assert oracle_mod.wfa(dele, s, pen)[1] == o + k * e  # text longer: I
        _, ops = oracle_mod.gotoh(s, dele, pen)
        assert ops.count("D") == k and "I" not in ops and "X" not in ops


def test_empty_sequences(oracle_mod):
    for pen in PENALTY_SETS:
        x, o, e = pen
        assert oracle_mod.wfa("", "", pen) == (0, 0, "")
        for L in (1, 5, 33):
            s = "ACGT" * 9
            s = s[:L]
            assert oracle_mod.wfa("", s, pen) == (0, o + L * e, "I" * L)
            assert oracle_mod.wfa(s, "", pen) == (0, o + L * e, "D" * L)
            assert oracle_mod.gotoh("", s, pen) == (o + L * e, "I" * L)


def test_symmetry_and_rescoring(oracle_mod):
    """score(P, T) == score(T, P); the swapped alignment with I and D
    exchanged rescores to that score; every alignment consumes n and m."""
    from paper_2204_02085_gb300 import synth

    b = synth.uniform_reads(300, 100, 4, seed=21)
    for pen in PENALTY_SETS:
        for i in range(0, 300, 3):
            p, t = b.pair(i)
            _, s1, ops1 = oracle_mod.wfa(p, t, pen)
            _, s2, ops2 = oracle_mod.wfa(t, p, pen)
            assert s1 == s2
            assert oracle_mod.rescore(t, p, swap_id(ops1), pen) == s1
            assert oracle_mod.rescore(p, t, swap_id(ops2), pen) == s2
            assert oracle_mod.rescore(p, t, ops1, pen) == s1
            assert sum(c in "MXD" for c in ops1) == len(p)
            assert sum(c in "MXI" for c in ops1) == len(t)


def test_gotoh_equals_wfa_on_paper_shaped_reads(oracle_mod):
    """100 bp pairs with 2 and 4 edits (the paper's E = 2 % / 4 % shape): the
    DP and the wavefront algorithm give the same score and, under the same
    tie-break, the same alignment."""
    from paper_2204_02085_gb300 import synth

    for edits, seed in ((2, 0), (4, 1), (10, 2)):
        b = synth.uniform_reads(400, 100, edits, seed=seed)
        for pen in PENALTY_SETS:
            for i in range(0, 400, 4):
                p, t = b.pair(i)
                gs, gops = oracle_mod.gotoh(p, t, pen)
                st, ws, wops = oracle_mod.wfa(p, t, pen)
                assert gs == ws and gops == wops


def test_unrelated_sequences(oracle_mod):
    from paper_2204_02085_gb300 import synth

    b = synth.random_pairs(60, 0, 80, seed=5)
    for pen in PENALTY_SETS:
        for i in range(b.n):
            p, t = b.pair(i)
            gs, gops = oracle_mod.gotoh(p, t, pen)
            st, ws, wops = oracle_mod.wfa(p, t, pen)
            assert gs == ws and gops == wops
            assert oracle_mod.rescore(p, t, wops, pen) == ws


def test_max_score_boundary(oracle_mod):
    p, t = "ACGTACGTAC", "ACGAACGTTC"  # two substitutions
    pen = (4, 6, 2)
    assert oracle_mod.wfa(p, t, pen)[:2] == (0, 8)
    assert oracle_mod.wfa(p, t, pen, max_score=8)[:2] == (0, 8)  # equal: ok
    assert oracle_mod.wfa(p, t, pen, max_score=7)[:2] == (oracle_mod.SCORE_LIMIT, -1)
    assert oracle_mod.wfa(p, t, pen, max_score=0)[:2] == (0, 8)  # <= 0: unbounded


def test_case_folding_and_invalid(oracle_mod):
    pen = (4, 6, 2)
    assert oracle_mod.wfa("acgtN", "ACGTA", pen)[0] == oracle_mod.INVALID_CHAR
    assert oracle_mod.wfa("ACGT", "ACGU", pen)[0] == oracle_mod.INVALID_CHAR
    assert oracle_mod.wfa("acGt", "ACgT", pen) == (0, 0, "MMMM")


def _load_golden(name):
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            p, t, x, o, e, score, cigar = line.split()
            p = "" if p == "-" else p
            t = "" if t == "-" else t
            cigar = "" if cigar == "-" else cigar
            rows.append((p, t, (int(x), int(o), int(e)), int(score), cigar))
    return rows


def test_golden_tie_break_cases(oracle_mod):
    """Hand-derived cases (derivations in the fixture file)."""
    rows = _load_golden("tie_break_cases.txt")
    assert len(rows) >= 8
    for p, t, pen, score, cigar in rows:
        st, s, ops = oracle_mod.wfa(p, t, pen)
        assert s == score, (p, t, pen)
        assert oracle_mod.runs_to_cigar(oracle_mod.ops_to_runs(ops)) == cigar, (p, t, pen, ops)
        gs, gops = oracle_mod.gotoh(p, t, pen)
        assert (gs, gops) == (s, ops)


def test_pack2bit_format(oracle_mod):
    """The packed format: A=0 C=1 G=2 T=3, 32 bases per word, first base in
    the top two bits, zero tail, one zero pad word."""
    rc, w = oracle_mod.pack2bit("ACGT")
    assert rc == 0 and list(w) == [0x1B << 56, 0]
    rc, w = oracle_mod.pack2bit("acgt" * 8 + "T")
    assert rc == 0 and len(w) == 3
    assert int(w[0]) == int("1B" * 8, 16) and int(w[1]) == 3 << 62 and int(w[2]) == 0
    rc, w = oracle_mod.pack2bit("")
    assert rc == 0 and list(w) == [0]
    assert oracle_mod.pack2bit("ACNT")[0] == -1
    # unpacking returns the input (upper-cased)
    rng = random.Random(9)
    for L in (1, 31, 32, 33, 64, 100, 257):
        s = "".join(rng.choice("ACGTacgt") for _ in range(L))
        rc, w = oracle_mod.pack2bit(s)
        back = "".join("ACGT"[(int(w[i // 32]) >> (62 - 2 * (i % 32))) & 3] for i in range(L))
        assert rc == 0 and back == s.upper()
        assert len(w) == (L + 31) // 32 + 1 and int(w[-1]) == 0
        tail = L % 32
        if tail:
            assert int(w[L // 32]) & ((1 << (64 - 2 * tail)) - 1) == 0


def test_batch_matches_single(oracle_mod):
    from paper_2204_02085_gb300 import synth

    b = synth.uniform_reads(500, 100, 4, seed=3)
    pen = (4, 6, 2)
    s, st, words, off = oracle_mod.wfa_batch(b, pen, nthreads=3)
    for i in range(0, 500, 7):
        p, t = b.pair(i)
        _, sc, ops = oracle_mod.wfa(p, t, pen)
        assert s[i] == sc and st[i] == 0
        assert oracle_mod.runs_to_ops(words[off[i]:off[i + 1]]) == ops
    s1, st1, w1, o1 = oracle_mod.wfa_batch(b, pen, nthreads=1)
    assert np.array_equal(s, s1) and np.array_equal(st, st1)
    assert np.array_equal(words, w1) and np.array_equal(off, o1)


# ------------------------------------------------------------ ends-free

ENDS_PENALTIES = [(4, 6, 2), (1, 0, 1), (2, 3, 1), (3, 0, 2)]


def check_ends(oracle, p, t, pen, ends):
    bs, _, _ = oracle.brute(p, t, pen, ends=ends)
    gs, gops = oracle.gotoh(p, t, pen, ends=ends)
    st, ws, wops = oracle.wfa(p, t, pen, ends=ends)
    assert st == oracle.OK
    assert bs == gs == ws, (p, t, pen, ends, bs, gs, ws)
    assert wops == gops, (p, t, pen, ends, gops, wops)
    assert oracle.rescore(p, t, wops, pen, ends=ends) == ws
    return ws, wops


@pytest.mark.parametrize("pen", ENDS_PENALTIES)
def test_ends_free_brute_force(oracle_mod, pen):
    """Free leading / trailing pattern and text characters: brute force over
    every alignment (scored with the free ends), Gotoh with free start and
    end cells, and WFA with a widened first wavefront and an end test over
    the free diagonals agree on the score; the two walk-backs give the same
    alignment, which rescores to that score."""
    rng = random.Random(sum(pen) * 31 + 7)
    for _ in range(700):
        p = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 6)))
        t = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 6)))
        ends = tuple(rng.randint(0, 4) for _ in range(4))
        check_ends(oracle_mod, p, t, pen, ends)
    for _ in range(300):  # repeats: many ties
        p = "".join(rng.choice("AC") for _ in range(rng.randint(0, 6)))
        t = "".join(rng.choice("AC") for _ in range(rng.randint(0, 6)))
        ends = tuple(rng.randint(0, 3) for _ in range(4))
        check_ends(oracle_mod, p, t, pen, ends)


def test_ends_free_zero_is_global(oracle_mod):
    rng = random.Random(3)
    for _ in range(300):
        p = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 12)))
        t = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 12)))
        for pen in PENALTY_SETS:
            assert oracle_mod.wfa(p, t, pen, ends=(0, 0, 0, 0)) == oracle_mod.wfa(p, t, pen)


def test_ends_free_everything_free(oracle_mod):
    """Every character may be skipped: the score is 0."""
    rng = random.Random(4)
    for _ in range(200):
        p = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 20)))
        t = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 20)))
        ends = (len(p), len(p), len(t), len(t))
        assert oracle_mod.wfa(p, t, (4, 6, 2), ends=ends)[1] == 0
        assert oracle_mod.gotoh(p, t, (4, 6, 2), want_ops=False, ends=ends)[0] == 0


def test_ends_free_semi_global_is_sellers(oracle_mod):
    """Text ends free, pattern global, unit costs: the score is the least edit
    distance between the pattern and any substring of the text (Sellers'
    textbook DP, written here)."""

    def sellers(a, b):
        prev = [0] * (len(b) + 1)  # any text prefix may be skipped
        for i in range(1, len(a) + 1):
            cur = [i] + [0] * len(b)
            for j in range(1, len(b) + 1):
                cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + (a[i - 1] != b[j - 1]))
            prev = cur
        return min(prev)  # any text suffix may be skipped

    rng = random.Random(5)
    for _ in range(400):
        p = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 10)))
        t = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 30)))
        ends = (0, 0, len(t), len(t))
        st, s, ops = oracle_mod.wfa(p, t, (1, 0, 1), ends=ends)
        assert s == sellers(p, t), (p, t)
        assert oracle_mod.gotoh(p, t, (1, 0, 1), want_ops=False, ends=ends)[0] == s
        assert oracle_mod.rescore(p, t, ops, (1, 0, 1), ends=ends) == s


def test_ends_free_swap_symmetry(oracle_mod):
    """Swapping pattern and text (and their free lengths) keeps the score."""
    rng = random.Random(6)
    for _ in range(300):
        p = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 15)))
        t = "".join(rng.choice("ACGT") for _ in range(rng.randint(0, 15)))
        pb, pe, tb, te = (rng.randint(0, 5) for _ in range(4))
        a = oracle_mod.wfa(p, t, (4, 6, 2), ends=(pb, pe, tb, te))[1]
        b = oracle_mod.wfa(t, p, (4, 6, 2), ends=(tb, te, pb, pe))[1]
        assert a == b


def test_ends_free_worked_examples(oracle_mod):
    """Hand-derived: a pattern that occurs inside the text aligns at cost 0
    with the flanks as free I runs; a pattern with a 3-base junk prefix and 2
    free pattern-begin characters pays one 1-base deletion (o + e)."""
    st, s, ops = oracle_mod.wfa("GATTA", "CCGATTACC", (4, 6, 2), ends=(0, 0, 9, 9))
    assert s == 0 and ops == "II" + "M" * 5 + "II"
    st, s, ops = oracle_mod.wfa("TTTGATTACA", "GATTACA", (4, 6, 2), ends=(2, 0, 0, 0))
    assert s == 8 and ops == "DDD" + "M" * 7
