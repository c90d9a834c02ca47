"""The oracle's work counters, which the benchmark's roofline model is built
on, pinned on hand-counted cases (penalties x=4, o=6, e=2; scores s = 0, 1,
2, ... unscaled, a wavefront counted only when one of its offsets exists).

  cells          sum over existing wavefronts of hi - lo + 1
  wavefronts     number of existing wavefronts
  char_compares  character comparisons made by extend (a stop at a sequence
                 end compares nothing)
  bt_steps       state visits of the backtrace, the final one at score 0
                 included

Each case's derivation is written beside it.
"""

import pytest

PEN = (4, 6, 2)


def counts_of(oracle_mod, p, t, pen=PEN):
    c = oracle_mod.Counts()
    rc, score, ops = oracle_mod.wfa(p, t, pen, counts=c)
    assert rc == 0
    return score, ops, (c.cells, c.wavefronts, c.char_compares, c.bt_steps)


def test_identical(oracle_mod):
    # s = 0: diagonal 0 only (1 cell); extend compares h = 0..3 (all match)
    # and stops at the text end h = 4 without a compare: 4 compares; the end
    # cell is reached at s = 0; the backtrace visits (M, 0) once.
    assert counts_of(oracle_mod, "AAAA", "AAAA") == (0, "MMMM", (1, 1, 4, 1))


def test_one_deletion(oracle_mod):
    # P = AAAA, T = AAA (k_f = -1).  s = 0: M_0[0] = 3 after 3 matching
    # compares (stop at h = m).  s = 2..6: every candidate is null or past an
    # end (M_4[0] + 1 = 4 > m), no wavefront.  s = 8: diagonals -1..1 from
    # M_0 (o + e = 8): D_8[-1] = M_0[0] = 3 (v = 4 = n: extend compares
    # nothing), the other two cells null: 3 cells, and M_8[-1] = 3 = m ends.
    # Backtrace: (M, 8, -1) picks D; (D, 8, -1) opens from M_0[0]; (M, 0)
    # emits 3 M: 3 visits.  Cells 1 + 3, wavefronts 2, compares 3.
    assert counts_of(oracle_mod, "AAAA", "AAA") == (8, "MMMD", (4, 2, 3, 3))


def test_one_substitution(oracle_mod):
    # P = ACGT, T = AGGT.  s = 0: A = A, C != G: 2 compares, M_0[0] = 1.
    # s = 4: only the mismatch source M_0[0] exists: diagonal 0, 1 cell,
    # M_4[0] = 2, then G = G, T = T and the text end: 2 compares, M_4[0] =
    # 4 = m ends.  Backtrace: (M, 4, 0) picks X; (M, 0) emits 1 M: 2 visits.
    assert counts_of(oracle_mod, "ACGT", "AGGT") == (4, "MXMM", (2, 2, 4, 2))


def test_empty_pattern(oracle_mod):
    # P = "", T = AC (k_f = 2).  s = 0: diagonal 0, v = 0 = n: no compare.
    # Wavefronts appear at s = 8 (I_8[1] = 1 from M_0[0]: diagonals -1..1,
    # 3 cells) and s = 10 (I_10[2] = 2 extending I_8[1]: diagonals -2..2,
    # 5 cells; M_10[2] = 2 = m ends).  Backtrace: (M, 10, 2) picks I;
    # (I, 10, 2) extends; (I, 8, 1) opens from M_0[0]; (M, 0) with h = 0:
    # 4 visits.  Cells 1 + 3 + 5 = 9, wavefronts 3, compares 0.
    assert counts_of(oracle_mod, "", "AC") == (10, "II", (9, 3, 0, 4))


@pytest.mark.parametrize("n", [1, 7, 33, 100])
def test_identical_lengths(oracle_mod, n):
    # identical sequences of n bases: one cell, n compares, one visit
    s = ("ACGT" * 40)[:n]
    assert counts_of(oracle_mod, s, s)[2] == (1, 1, n, 1)
