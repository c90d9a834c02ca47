"""Planted mistakes in a copy of the oracle must fail the pins.

Each mutant below changes one line of ``oracle/wfa_oracle.c`` the way a
plausible slip would (a dropped term, a wrong index or sign, a swapped
priority, a missing bound).  The mutant is compiled on the CPU into a
temporary library and run in a child process against a reduced pin suite
(brute force, Levenshtein, closed forms); the test passes only if the suite
reports a failure (or the child crashes).  The unmutated oracle must pass the
same suite.
"""

import ctypes
import os
import random
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "wfa_oracle.c")

MUTANTS = {
    "wfa_I_drops_plus_one": ("          iv += 1;\n          if (iv > m) iv = NUL;",
                             "          iv += 0;\n          if (iv > m) iv = NUL;"),
    "wfa_D_wrong_diagonal": ("int64_t dv = max_non_null(wf_get(wf, so, k + 1, 'M'),",
                             "int64_t dv = max_non_null(wf_get(wf, so, k - 1, 'M'),"),
    "wfa_X_bound_wrong_sign": ("          xv += 1;\n          if (xv > m || xv - k > n) xv = NUL;\n        }\n        int64_t mv",
                               "          xv += 1;\n          if (xv > m || xv + k > n) xv = NUL;\n        }\n        int64_t mv"),
    "wfa_tie_I_before_X": ("if (xv != NUL && (iv == NUL || xv >= iv) && (dv == NUL || xv >= dv))",
                           "if (xv != NUL && (iv == NUL || xv > iv) && (dv == NUL || xv >= dv))"),
    "wfa_gap_open_before_extend": ("if (wf_get(wf, s - e, k - 1, 'I') == h - 1) {",
                                   "if (0) {"),
    "wfa_wrong_final_diagonal": ("int64_t kf = m - n;", "int64_t kf = n - m;"),
    "wfa_extend_short_by_one": ("while (h - k < n && h < m) {", "while (h - k < n - 1 && h < m) {"),
    "wfa_range_missing_minus_one": ("if (wf[so].lo - 1 < lo) lo = wf[so].lo - 1;",
                                    "if (wf[so].lo - 1 < lo) lo = wf[so].lo;"),
    "wfa_extend_gap_sign": ("        if (dv != NUL && dv - k > n) dv = NUL;",
                            "        if (dv != NUL && dv + k > n) dv = NUL;"),
    "gotoh_open_without_e": ("if (h > 0) iv = min2(AT(H, v, h - 1) + o + e, AT(I, v, h - 1) + e);",
                             "if (h > 0) iv = min2(AT(H, v, h - 1) + o, AT(I, v, h - 1) + e);"),
    "gotoh_walkback_match_first": ("        if (v > 0 && h > 0 && !same(P, v - 1, T, h - 1) &&\n            AT(H, v - 1, h - 1) + x == s) {",
                                   "        if (v > 0 && h > 0 && !same(P, v - 1, T, h - 1) &&\n            AT(H, v - 1, h - 1) + x == s && 0) {"),
    "rescore_open_costs_e": ("      cost += (prev == 'I') ? e : o + e;", "      cost += e;"),
    "lex_rank_D_before_I": ("    case 'I': return 2;\n    case 'D': return 3;",
                            "    case 'I': return 3;\n    case 'D': return 2;"),
}


def _levenshtein(a, b):
    prev = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        cur = [i] + [0] * len(b)
        for j in range(1, len(b) + 1):
            cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + (a[i - 1] != b[j - 1]))
        prev = cur
    return prev[-1]


def pin_suite(so_path):
    """Run a reduced pin suite against the oracle library at so_path; return
    the number of failed checks."""
    L = ctypes.CDLL(so_path)
    i64, cp, vp = ctypes.c_int64, ctypes.c_char_p, ctypes.c_void_p
    L.oracle_brute.argtypes = [cp, ctypes.c_int, cp, ctypes.c_int, i64, i64, i64, vp, vp, vp]
    L.oracle_brute.restype = i64
    L.oracle_gotoh.argtypes = [cp, i64, cp, i64, i64, i64, i64, vp, vp]
    L.oracle_gotoh.restype = i64
    L.oracle_wfa.argtypes = [cp, i64, cp, i64, i64, i64, i64, i64, ctypes.c_int, vp, vp, i64, vp, vp]
    L.oracle_wfa.restype = ctypes.c_int

    def brute(p, t, pen):
        buf = ctypes.create_string_buffer(32)
        nops = ctypes.c_int64()
        c = L.oracle_brute(p, len(p), t, len(t), *pen, ctypes.cast(buf, vp), ctypes.byref(nops), None)
        return c, buf.raw[: nops.value]

    def gotoh(p, t, pen):
        buf = ctypes.create_string_buffer(len(p) + len(t) + 1)
        nops = ctypes.c_int64()
        c = L.oracle_gotoh(p, len(p), t, len(t), *pen, ctypes.cast(buf, vp), ctypes.byref(nops))
        return c, buf.raw[: nops.value]

    def wfa(p, t, pen):
        cap = len(p) + len(t) + 1
        buf = ctypes.create_string_buffer(cap)
        nops, sc = ctypes.c_int64(), ctypes.c_int64()
        # 1000 is far above any optimal score of these short inputs, so a
        # mutant that never reaches the end stops with a score-limit status
        rc = L.oracle_wfa(p, len(p), t, len(t), *pen, 1000, 1, ctypes.byref(sc),
                          ctypes.cast(buf, vp), cap, ctypes.byref(nops), None)
        return rc, sc.value, buf.raw[: nops.value]

    fails = 0
    rng = random.Random(1)
    cases = [(b"", b""), (b"A", b""), (b"", b"ACG"), (b"AAAA", b"AAA"), (b"A", b"C"),
             (b"GATTACA", b"GATACA"), (b"ACGT", b"ACGT"), (b"ACT", b"ACGT")]
    for _ in range(250):
        cases.append((bytes(rng.choice(b"ACGT") for _ in range(rng.randint(0, 5))),
                      bytes(rng.choice(b"ACGT") for _ in range(rng.randint(0, 5)))))
    for pen in ((4, 6, 2), (16, 6, 2), (1, 0, 1), (5, 1, 1)):
        for p, t in cases:
            bs, bops = brute(p, t, pen)
            gs, gops = gotoh(p, t, pen)
            rc, ws, wops = wfa(p, t, pen)
            if rc != 0 or not (bs == gs == ws) or not (bops == gops == wops):
                fails += 1
            if pen == (1, 0, 1) and bs != _levenshtein(p, t):
                fails += 1
            if p == t and (ws != 0 or wops != b"M" * len(p)):
                fails += 1
    # longer closed forms: one gap of length k costs o + k e
    for pen in ((4, 6, 2), (2, 3, 1)):
        for _ in range(40):
            s = bytes(rng.choice(b"ACGT") for _ in range(rng.randint(5, 40)))
            k = rng.randint(1, 4)
            j = rng.randint(0, len(s) - k)
            d = s[:j] + s[j + k:]
            if wfa(s, d, pen)[1] != pen[1] + k * pen[2] or gotoh(d, s, pen)[0] != pen[1] + k * pen[2]:
                fails += 1
    return fails


def _build(src_text, out_dir, name):
    c = os.path.join(out_dir, name + ".c")
    so = os.path.join(out_dir, name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", so, c, "-lpthread"])
    return so


def _run_suite(so):
    """Failures reported by the child, or None if it crashed, ran out of its
    memory cap or did not finish in time (a mutant that never terminates)."""
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), so],
                           capture_output=True, text=True, timeout=30)
    except subprocess.TimeoutExpired:
        return None
    if r.returncode != 0:
        return None
    return int(r.stdout.strip().splitlines()[-1])


def test_unmutated_oracle_passes_reduced_suite(tmp_path):
    with open(SRC) as f:
        src = f.read()
    so = _build(src, str(tmp_path), "orig")
    assert _run_suite(so) == 0


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    with open(SRC) as f:
        src = f.read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, "mutation site not unique: " + name
    so = _build(src.replace(old, new), str(tmp_path), name)
    fails = _run_suite(so)
    assert fails is None or fails > 0, "mutant %s survived the pins" % name


if __name__ == "__main__":
    import resource

    # a mutant that never reaches the end keeps allocating wavefronts: cap it
    resource.setrlimit(resource.RLIMIT_AS, (1 << 31, 1 << 31))
    print(pin_suite(sys.argv[1]))
