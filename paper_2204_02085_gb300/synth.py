"""Seeded synthetic read pairs shaped like the paper's workloads.

This module holds no alignment arithmetic: it only draws random sequences and
applies random edits.  Both the CUDA path's tests/benchmark and the CPU oracle
consume its output, which is why it lives on its own.

The paper (Sec. II) aligns 5 million pairs of 100 bp reads at edit-distance
thresholds E = 2 % and 4 %; its read set is not available, so these pairs
stand in for it with the same shape:

* text    = ``length`` bases drawn uniformly from {A, C, G, T};
* pattern = the text after ``n_edits`` edits applied one after another to a
  copy of it; each edit is a substitution, an insertion or a deletion with
  probability 1/3 each, at a uniform position of the current sequence
  (``len + 1`` slots for an insertion); a substitution picks one of the three
  other bases uniformly, an insertion draws a uniform base.  Edits may
  overlap; the optimal score is computed, never assumed from the edit count.

Random numbers come from ``numpy.random.Generator(PCG64(seed))``.  Pairs are
produced in chunks of ``CHUNK`` pairs; within a chunk the draws are, in order:
the text bases, then per edit step the edit kind, a uniform position variate,
the substitution offset (1..3) and the inserted base, each as one array over
the chunk's pairs.  The output is therefore a pure function of the arguments.
"""

from __future__ import annotations

import dataclasses
import hashlib

import numpy as np

CHUNK = 1 << 18
ALPHABET = np.frombuffer(b"ACGT", dtype=np.uint8)


@dataclasses.dataclass
class Batch:
    """Concatenated ASCII sequences with per-pair offsets and lengths."""

    patterns: np.ndarray  # uint8, concatenated
    pattern_offsets: np.ndarray  # int64 [n]
    pattern_lengths: np.ndarray  # int32 [n]
    texts: np.ndarray  # uint8, concatenated
    text_offsets: np.ndarray  # int64 [n]
    text_lengths: np.ndarray  # int32 [n]

    @property
    def n(self) -> int:
        return int(self.pattern_lengths.shape[0])

    def pair(self, i: int) -> tuple[bytes, bytes]:
        po, pl = int(self.pattern_offsets[i]), int(self.pattern_lengths[i])
        to, tl = int(self.text_offsets[i]), int(self.text_lengths[i])
        return self.patterns[po:po + pl].tobytes(), self.texts[to:to + tl].tobytes()

    def subset(self, idx) -> "Batch":
        """A new back-to-back batch holding the pairs ``idx`` in that order."""
        idx = np.asarray(idx, dtype=np.int64)
        return from_pairs([self.pair(int(i)) for i in idx])

    def sha256(self) -> str:
        h = hashlib.sha256()
        for a in (self.patterns, self.pattern_offsets, self.pattern_lengths,
                  self.texts, self.text_offsets, self.text_lengths):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()


def _concat(rows: np.ndarray, lengths: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    width = rows.shape[1]
    mask = np.arange(width)[None, :] < lengths[:, None]
    flat = np.ascontiguousarray(rows[mask])
    offsets = np.zeros(len(lengths), dtype=np.int64)
    if len(lengths) > 1:
        np.cumsum(lengths[:-1], out=offsets[1:])
    return flat, offsets


def _edit_chunk(rng: np.random.Generator, texts: np.ndarray, n_edits: int):
    """Apply n_edits sequential random edits to each row of texts (codes
    0..3).  Returns (rows, lengths) of the edited copies."""
    npairs, length = texts.shape
    width = length + n_edits + 1
    rows = np.zeros((npairs, width), dtype=np.uint8)
    rows[:, :length] = texts
    lens = np.full(npairs, length, dtype=np.int64)
    cols = np.arange(width)[None, :]
    r = np.arange(npairs)
    for _ in range(n_edits):
        kind = rng.integers(0, 3, size=npairs)  # 0 sub, 1 ins, 2 del
        u = rng.random(size=npairs)
        delta = rng.integers(1, 4, size=npairs).astype(np.uint8)
        ins_base = rng.integers(0, 4, size=npairs).astype(np.uint8)
        slots = lens + (kind == 1)
        pos = np.minimum((u * slots).astype(np.int64), slots - 1)
        # a deletion or substitution needs a base to act on
        empty = lens == 0
        kind = np.where(empty, 1, kind)
        pos = np.where(empty, 0, pos)
        sub = kind == 0
        if sub.any():
            rs, ps = r[sub], pos[sub]
            rows[rs, ps] = (rows[rs, ps] + delta[sub]) % 4
        ins = kind == 1
        if ins.any():
            ri = rows[ins]
            pi = pos[ins][:, None]
            shifted = np.roll(ri, 1, axis=1)
            ri = np.where(cols < pi, ri, np.where(cols == pi, ins_base[ins][:, None], shifted))
            rows[ins] = ri
            lens[ins] += 1
        dele = kind == 2
        if dele.any():
            rd = rows[dele]
            pd = pos[dele][:, None]
            shifted = np.roll(rd, -1, axis=1)
            rd = np.where(cols < pd, rd, shifted)
            rows[dele] = rd
            lens[dele] -= 1
        # keep the tail past each row's length zeroed
        rows[cols >= lens[:, None]] = 0
    return rows, lens


def uniform_reads(n_pairs: int, length: int = 100, n_edits: int = 2, seed: int = 0) -> Batch:
    """``n_pairs`` pairs: text = ``length`` uniform bases, pattern = text with
    exactly ``n_edits`` sequential edits (see the module docstring)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pats, plens, txts, tlens = [], [], [], []
    done = 0
    while done < n_pairs:
        c = min(CHUNK, n_pairs - done)
        codes = rng.integers(0, 4, size=(c, length)).astype(np.uint8)
        rows, lens = _edit_chunk(rng, codes, n_edits)
        pats.append(ALPHABET[rows][np.arange(rows.shape[1])[None, :] < lens[:, None]])
        plens.append(lens.astype(np.int32))
        txts.append(ALPHABET[codes].reshape(-1))
        tlens.append(np.full(c, length, dtype=np.int32))
        done += c
    plen = np.concatenate(plens) if plens else np.zeros(0, np.int32)
    tlen = np.concatenate(tlens) if tlens else np.zeros(0, np.int32)
    patterns = np.ascontiguousarray(np.concatenate(pats)) if pats else np.zeros(0, np.uint8)
    texts = np.ascontiguousarray(np.concatenate(txts)) if txts else np.zeros(0, np.uint8)
    poff = np.zeros(len(plen), dtype=np.int64)
    toff = np.zeros(len(tlen), dtype=np.int64)
    if len(plen) > 1:
        np.cumsum(plen[:-1], out=poff[1:])
        np.cumsum(tlen[:-1], out=toff[1:])
    return Batch(patterns, poff, plen, texts, toff, tlen)


def random_pairs(n_pairs: int, min_len: int, max_len: int, seed: int,
                 edit_rate: float | None = None, alphabet: bytes = b"ACGT") -> Batch:
    """Pairs with independent uniform lengths in [min_len, max_len].  With
    ``edit_rate`` None the two sequences are unrelated; otherwise the pattern
    is the text after round(edit_rate * len) edits as in ``uniform_reads``.
    ``alphabet`` may include lowercase letters to exercise case folding."""
    rng = np.random.Generator(np.random.PCG64(seed))
    alpha = np.frombuffer(alphabet, dtype=np.uint8)
    pairs = []
    for _ in range(n_pairs):
        tl = int(rng.integers(min_len, max_len + 1))
        t = alpha[rng.integers(0, len(alpha), size=tl)]
        if edit_rate is None:
            pl = int(rng.integers(min_len, max_len + 1))
            p = alpha[rng.integers(0, len(alpha), size=pl)]
        else:
            codes = rng.integers(0, 4, size=(1, tl)).astype(np.uint8)
            rows, lens = _edit_chunk(rng, codes, int(round(edit_rate * tl)))
            t = ALPHABET[codes[0]]
            p = ALPHABET[rows[0, : int(lens[0])]]
        pairs.append((p.tobytes(), t.tobytes()))
    return from_pairs(pairs)


def _edit_one_pass(rng: np.random.Generator, text: np.ndarray, k: int) -> np.ndarray:
    """Pattern from text (codes 0..3) with k edit events in one left-to-right
    pass: k positions drawn uniformly over the text (with replacement); each
    event is a substitution (one of the three other bases), a deletion of the
    base there, or an insertion of a uniform base before it, 1/3 each.
    Draw order: positions, kinds, substitution offsets, inserted bases."""
    L = len(text)
    if k == 0 or L == 0:
        return text.copy()
    pos = np.sort(rng.integers(0, L, size=k))
    kind = rng.integers(0, 3, size=k)
    delta = rng.integers(1, 4, size=k).astype(np.uint8)
    ins = rng.integers(0, 4, size=k).astype(np.uint8)
    pat = text.copy()
    sub = kind == 0
    np.add.at(pat, pos[sub], delta[sub])
    pat %= 4
    keep = np.ones(L, dtype=bool)
    keep[pos[kind == 2]] = False
    ip = pos[kind == 1]
    out = np.insert(pat, ip, ins[kind == 1])
    return out[np.insert(keep, ip, True)]


def _pairs_from_codes(texts, pats) -> Batch:
    tl = np.array([len(t) for t in texts], dtype=np.int32)
    pl = np.array([len(p) for p in pats], dtype=np.int32)
    txt = ALPHABET[np.concatenate(texts)] if texts else np.zeros(0, np.uint8)
    pat = ALPHABET[np.concatenate(pats)] if pats else np.zeros(0, np.uint8)
    poff = np.zeros(len(pl), dtype=np.int64)
    toff = np.zeros(len(tl), dtype=np.int64)
    if len(pl) > 1:
        np.cumsum(pl[:-1], out=poff[1:])
        np.cumsum(tl[:-1], out=toff[1:])
    return Batch(np.ascontiguousarray(pat), poff, pl, np.ascontiguousarray(txt), toff, tl)


def long_reads(n_pairs: int, length: int = 10_000, rate_lo: float = 0.01, rate_hi: float = 0.05,
               seed: int = 4) -> Batch:
    """Long-read pairs: text = `length` uniform bases; pattern = text after
    round(r * length) one-pass edit events, r ~ U[rate_lo, rate_hi] per pair
    (see _edit_one_pass).  Per pair the draws are: text, r, then the edits."""
    rng = np.random.Generator(np.random.PCG64(seed))
    texts, pats = [], []
    for _ in range(n_pairs):
        t = rng.integers(0, 4, size=length).astype(np.uint8)
        k = int(round(rng.uniform(rate_lo, rate_hi) * length))
        texts.append(t)
        pats.append(_edit_one_pass(rng, t, k))
    return _pairs_from_codes(texts, pats)


def mixed_reads(n_pairs: int, len_lo: int = 100, len_hi: int = 2000, rate_hi: float = 0.10,
                repeat_frac: float = 0.05, seed: int = 3, rate_lo: float = 0.0) -> Batch:
    """Pairs of uneven length and divergence: text length log-uniform in
    [len_lo, len_hi], edit rate r ~ U[rate_lo, rate_hi]; a fraction repeat_frac of
    the texts carry a tandem repeat (a uniform 50-mer repeated u ~ U{2..6}
    times, written over a uniform window of the text, clipped at its end)
    before the one-pass edits.  Per pair the draws are: length, text, the
    repeat coin (and repeat unit, count, start), r, then the edits."""
    rng = np.random.Generator(np.random.PCG64(seed))
    texts, pats = [], []
    lo, hi = np.log(len_lo), np.log(len_hi)
    for _ in range(n_pairs):
        L = int(round(np.exp(rng.uniform(lo, hi))))
        t = rng.integers(0, 4, size=L).astype(np.uint8)
        if rng.random() < repeat_frac:
            unit = rng.integers(0, 4, size=50).astype(np.uint8)
            rep = np.tile(unit, int(rng.integers(2, 7)))
            start = int(rng.integers(0, L))
            span = min(len(rep), L - start)
            t[start:start + span] = rep[:span]
        k = int(round(rng.uniform(rate_lo, rate_hi) * L))
        texts.append(t)
        pats.append(_edit_one_pass(rng, t, k))
    return _pairs_from_codes(texts, pats)


def from_pairs(pairs) -> Batch:
    """Back-to-back batch from a list of (pattern bytes, text bytes)."""
    pl = np.array([len(p) for p, _ in pairs], dtype=np.int32)
    tl = np.array([len(t) for _, t in pairs], dtype=np.int32)
    pat = np.frombuffer(b"".join(p for p, _ in pairs), dtype=np.uint8).copy()
    txt = np.frombuffer(b"".join(t for _, t in pairs), dtype=np.uint8).copy()
    poff = np.zeros(len(pl), dtype=np.int64)
    toff = np.zeros(len(tl), dtype=np.int64)
    if len(pl) > 1:
        np.cumsum(pl[:-1], out=poff[1:])
        np.cumsum(tl[:-1], out=toff[1:])
    return Batch(pat, poff, pl, txt, toff, tl)


def reads_in_windows(n_pairs: int, read_len: int = 100, flank: int = 100, n_edits: int = 3,
                     seed: int = 6) -> Batch:
    """Reads against reference windows (the shape of ends-free / semi-global
    alignment): pattern = `read_len` uniform bases; text = a uniform left
    flank of U{0..flank} bases + the read after `n_edits` sequential edits
    (the generator of uniform_reads) + a uniform right flank of U{0..flank}
    bases.  Draws: the uniform_reads batch (seed), then from PCG64(seed + 1)
    the left flank lengths, the right flank lengths, the left flank bases and
    the right flank bases, each as one array."""
    core = uniform_reads(n_pairs, read_len, n_edits, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    left = rng.integers(0, flank + 1, size=n_pairs).astype(np.int64)
    right = rng.integers(0, flank + 1, size=n_pairs).astype(np.int64)
    lb = ALPHABET[rng.integers(0, 4, size=int(left.sum()))]
    rb = ALPHABET[rng.integers(0, 4, size=int(right.sum()))]
    el = core.pattern_lengths.astype(np.int64)  # the edited read (uniform_reads' pattern)
    tl = left + el + right
    toff = np.zeros(n_pairs, dtype=np.int64)
    if n_pairs > 1:
        np.cumsum(tl[:-1], out=toff[1:])
    txt = np.empty(int(tl.sum()), dtype=np.uint8)

    def place(dst_start, src, lengths):
        src_off = np.zeros(n_pairs, dtype=np.int64)
        if n_pairs > 1:
            np.cumsum(lengths[:-1], out=src_off[1:])
        pos = np.repeat(dst_start - src_off, lengths) + np.arange(int(lengths.sum()), dtype=np.int64)
        txt[pos] = src

    place(toff, lb, left)
    place(toff + left, core.patterns, el)
    place(toff + left + el, rb, right)
    return Batch(np.ascontiguousarray(core.texts), core.text_offsets.copy(), core.text_lengths.copy(), txt, toff,
                 tl.astype(np.int32))
