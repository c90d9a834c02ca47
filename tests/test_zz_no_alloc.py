"""The entry point that allocates nothing (wfa_gpu_align_short_noalloc).

Some callers cannot call cudaMalloc: code running while a stream is being
captured into a CUDA graph, applications whose device memory belongs to a
pool that forbids foreign allocations, latency-critical paths.  For them
the library keeps the short-read path's scratch in one static device array.
This test calls that entry point through the C ABI, twice in a row on the
same inputs (the array keeps the first call's contents), and requires the
same scores, status, CIGAR offsets and CIGAR words as the regular entry
point, bit for bit (integer results; no tolerance).  It lives in a file
that pytest collects last, so a run that stops at the first failure has
run every other test before it.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev(t, a):
    return t.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _inputs():
    from paper_2204_02085_gb300 import synth

    a = synth.uniform_reads(3000, 100, 2, seed=11)
    b = synth.uniform_reads(3000, 100, 4, seed=12)
    edge = [(b"", b""), (b"ACGT", b""), (b"", b"acg"), (b"AAAA", b"AAA"), (b"ACGN", b"ACGT"),
            (b"A" * 127, b"C" * 2 + b"A" * 125), (b"acgtACGT" * 15, b"ACGTacgt" * 15)]
    pairs = [a.pair(i) for i in range(a.n)] + [b.pair(i) for i in range(b.n)] + edge
    return synth.from_pairs(pairs)


def test_noalloc_matches_align_batch_twice():
    import torch

    from paper_2204_02085_gb300 import build

    build.build()
    import paper_2204_02085_gb300 as pkg

    batch = _inputs()
    n = batch.n
    pen = (4, 6, 2)
    with pkg.Aligner(0) as al:
        ref = al.align(batch, pen)
    stream = torch.cuda.current_stream(torch.device("cuda:0"))
    pat, txt = _dev(torch, batch.patterns), _dev(torch, batch.texts)
    plen, tlen = _dev(torch, batch.pattern_lengths), _dev(torch, batch.text_lengths)
    poff, toff = _dev(torch, batch.pattern_offsets), _dev(torch, batch.text_offsets)
    cap = int(ref[3][-1])
    for with_offsets in (True, True, False):  # two calls in a row, then back-to-back offsets
        s = torch.full((n,), 12345, dtype=torch.int32, device="cuda:0")
        st = torch.full((n,), 99, dtype=torch.int8, device="cuda:0")
        off = torch.full((n + 1,), -5, dtype=torch.int64, device="cuda:0")
        w = torch.zeros(cap, dtype=torch.int32, device="cuda:0")
        rc = pkg.wfa_gpu_align_short_noalloc(
            stream.cuda_stream, n, pat.data_ptr(), poff.data_ptr() if with_offsets else None, plen.data_ptr(),
            txt.data_ptr(), toff.data_ptr() if with_offsets else None, tlen.data_ptr(), pen, 0, s.data_ptr(),
            st.data_ptr(), w.data_ptr(), cap, off.data_ptr())
        torch.cuda.synchronize()
        assert rc == pkg.WFA_GPU_OK, pkg.wfa_gpu_strerror(rc)
        assert np.array_equal(s.cpu().numpy(), ref[0])
        assert np.array_equal(st.cpu().numpy(), ref[1])
        assert np.array_equal(off.cpu().numpy(), ref[3])
        assert np.array_equal(w.cpu().numpy().view(np.uint32), ref[2])


def test_noalloc_rejects_sizes_beyond_its_limits():
    import torch

    import paper_2204_02085_gb300 as pkg
    from paper_2204_02085_gb300 import synth

    stream = torch.cuda.current_stream(torch.device("cuda:0")).cuda_stream
    dummy = torch.zeros(16, dtype=torch.int64, device="cuda:0").data_ptr()
    too_many = pkg.WFA_GPU_NOALLOC_MAX_PAIRS + 1
    rc = pkg.wfa_gpu_align_short_noalloc(stream, too_many, dummy, None, dummy, dummy, None, dummy, (4, 6, 2), 0,
                                         dummy, dummy, dummy, 0, dummy)
    assert rc == pkg.WFA_GPU_EINVAL
    long = synth.from_pairs([(b"A" * 128, b"A" * 128)])
    s = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    st = torch.zeros(1, dtype=torch.int8, device="cuda:0")
    off = torch.zeros(2, dtype=torch.int64, device="cuda:0")
    w = torch.zeros(4, dtype=torch.int32, device="cuda:0")
    rc = pkg.wfa_gpu_align_short_noalloc(stream, 1, _dev(torch, long.patterns).data_ptr(), None,
                                         _dev(torch, long.pattern_lengths).data_ptr(),
                                         _dev(torch, long.texts).data_ptr(), None,
                                         _dev(torch, long.text_lengths).data_ptr(), (4, 6, 2), 0, s.data_ptr(),
                                         st.data_ptr(), w.data_ptr(), 4, off.data_ptr())
    assert rc == pkg.WFA_GPU_EINVAL
