"""The plain path (WFA_GPU_PLAIN, the comparison baseline: fixed variant, no
autotuner, no longest-first order, no graph), the arena-only path
(WFA_GPU_ARENA_ONLY) and graph replay (WFA_GPU_GRAPH) give exactly the
results of the default path."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2204_02085_gb300 import build

    build.build()
    import paper_2204_02085_gb300 as p

    return p


def _mixed(seed, n):
    from paper_2204_02085_gb300 import synth

    a = synth.uniform_reads(n, 100, 3, seed=seed)
    b = synth.mixed_reads(n // 10, 100, 1500, 0.08, 0.05, seed=seed + 1)
    return synth.from_pairs([a.pair(i) for i in range(a.n)] + [b.pair(i) for i in range(b.n)])


def test_plain_path_matches(pkg, oracle_mod):
    batch = _mixed(70, 3000)
    with pkg.Aligner(0, 4 << 30) as al:
        ref = al.align(batch, (4, 6, 2))
        got = al.align(batch, (4, 6, 2), plain=True)
        for x, y in zip(ref, got):
            assert np.array_equal(x, y)
        so = al.align(batch, (4, 6, 2), plain=True, score_only=True)
        assert np.array_equal(so[0], ref[0]) and np.array_equal(so[1], ref[1])
        ao = al.align(batch, (4, 6, 2), arena_only=True)  # every pair on arena teams
        for x, y in zip(ref, ao):
            assert np.array_equal(x, y)
    want = oracle_mod.wfa_batch(batch, (4, 6, 2), nthreads=8)
    assert np.array_equal(ref[0], want[0]) and np.array_equal(ref[2], want[2])


class _Dev:
    """Device copies of a batch in fixed buffers (contents can be replaced)."""

    def __init__(self, torch, batch, cap):
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")
        self.pat, self.plen = t(batch.patterns), t(batch.pattern_lengths)
        self.txt, self.tlen = t(batch.texts), t(batch.text_lengths)
        n = batch.n
        self.s = torch.empty(n, dtype=torch.int32, device="cuda:0")
        self.st = torch.empty(n, dtype=torch.int8, device="cuda:0")
        self.off = torch.empty(n + 1, dtype=torch.int64, device="cuda:0")
        self.w = torch.empty(cap, dtype=torch.int32, device="cuda:0")

    def load(self, torch, batch):
        self.pat.copy_(torch.from_numpy(batch.patterns))
        self.txt.copy_(torch.from_numpy(batch.texts))
        self.plen.copy_(torch.from_numpy(batch.pattern_lengths))
        self.tlen.copy_(torch.from_numpy(batch.text_lengths))

    def out(self):
        off = self.off.cpu().numpy()
        return (self.s.cpu().numpy(), self.st.cpu().numpy(), self.w.cpu().numpy().view(np.uint32)[: int(off[-1])],
                off)


def _same_shape_batches(k):
    """k batches of equal sizes (pair count, every sequence length) and
    different contents."""
    from paper_2204_02085_gb300 import synth

    base = synth.uniform_reads(4000, 100, 0, seed=80)  # no edits: all lengths 100
    out = []
    rng = np.random.default_rng(81)
    for j in range(k):
        texts = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, size=base.texts.size)]
        pats = texts.copy()
        flip = rng.random(pats.size) < 0.02 * (j + 1)
        pats[flip] = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, size=int(flip.sum()))]
        out.append(synth.Batch(pats, base.pattern_offsets, base.pattern_lengths, texts, base.text_offsets,
                               base.text_lengths))
    return out


def test_graph_replay_follows_new_contents(pkg):
    import torch

    batches = _same_shape_batches(4)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s), pkg.Aligner(0) as al, pkg.Aligner(0) as ref:
        al.set_stream(s)
        d = _Dev(torch, batches[0], 16 * batches[0].n)
        for j, b in enumerate(batches + batches[:1]):
            d.load(torch, b)
            rc = al.align_device(d.pat, None, d.plen, d.txt, None, d.tlen, d.s, d.st, d.w, d.off, graph=True,
                                 timing=True)
            s.synchronize()
            assert rc == pkg.WFA_GPU_OK
            got = d.out()
            want = ref.align(b, (4, 6, 2))
            for x, y in zip(got, want):
                assert np.array_equal(x, y), j


def test_graph_replay_rejects_bad_lengths(pkg):
    import torch

    b = _same_shape_batches(1)[0]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s), pkg.Aligner(0) as al:
        al.set_stream(s)
        d = _Dev(torch, b, 16 * b.n)
        for _ in range(2):
            assert al.align_device(d.pat, None, d.plen, d.txt, None, d.tlen, d.s, d.st, d.w, d.off,
                                   graph=True) == pkg.WFA_GPU_OK
        s.synchronize()
        d.plen[7] = -3
        with pytest.raises(pkg.WfaGpuError) as ei:
            al.align_device(d.pat, None, d.plen, d.txt, None, d.tlen, d.s, d.st, d.w, d.off, graph=True)
        assert ei.value.code == pkg.WFA_GPU_EINVAL
        d.plen[7] = 100
        assert al.align_device(d.pat, None, d.plen, d.txt, None, d.tlen, d.s, d.st, d.w, d.off,
                               graph=True) == pkg.WFA_GPU_OK


def test_graph_replay_with_arena_retries(pkg, oracle_mod):
    """Replays whose deferred pairs outgrow their arena slices fall back to
    eager retries and still match."""
    import torch

    from paper_2204_02085_gb300 import synth

    b = synth.random_pairs(40, 300, 900, seed=90)  # unrelated: large wavefronts
    want = oracle_mod.wfa_batch(b, (4, 6, 2), nthreads=8)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s), pkg.Aligner(0, scratch_bytes=96 << 20) as al:
        al.set_stream(s)
        d = _Dev(torch, b, int(want[3][-1]) + 16)
        for _ in range(3):
            assert al.align_device(d.pat, None, d.plen, d.txt, None, d.tlen, d.s, d.st, d.w, d.off,
                                   graph=True) == pkg.WFA_GPU_OK
            s.synchronize()
            got = d.out()
            for x, y in zip(got, want):
                assert np.array_equal(x, y)


def test_work_balanced_shards_reassemble(pkg, oracle_mod):
    """One mixed-length batch split into work-balanced shares, each aligned by
    its own context (two contexts on GPU 0 stand in for two devices: their
    kernels never wait on each other), reassembled: the one-context result
    and the oracle's."""
    from paper_2204_02085_gb300 import sharding, synth

    batch = synth.mixed_reads(2000, 100, 2000, 0.10, 0.05, seed=90)
    got = sharding.align_multi_gpu(batch, (4, 6, 2), [0, 0], scratch_bytes=2 << 30)
    with pkg.Aligner(0, 2 << 30) as al:
        one = al.align(batch, (4, 6, 2))
    want = oracle_mod.wfa_batch(batch, (4, 6, 2), nthreads=16)
    for x, y, z in zip(got, one, want):
        assert np.array_equal(x, y) and np.array_equal(x, z)
