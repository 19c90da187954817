"""mh_solve_noalloc: the solve for callers that cannot allocate device memory.

Such callers (code running while another component owns all device memory
through its own pool, plug-ins handed fixed buffers, latency-critical streams
that must not see allocator traffic) get every piece of scratch from one fixed
__device__ array inside the library.  This file runs last so that a failure
here leaves every other test already run.  The entry point is called through
the C ABI and must return exactly what mh_solve returns, on consecutive calls
that reuse the shared scratch array.

Cases: h = 1 (no leaf phase), h = 2 and 3, h = 4 (the third frontier region), a
cohort at the largest gene count the scratch holds (G = 8192: the full width of
the one-block key sort, and depth-1 regions filled to their exact capacity), and
a dense cohort whose depth-2 frontier passes the fixed 2^17-prefix limit, which
must return MH_ENOMEM naming the limit and leave the next call correct.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

ALPHA = (1, 10)


def _lib():
    pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_16721_gb300 import mh
    return mh


def _cohorts():
    small = synth.generate(synth.c2_law(900, 190, 70, seed=21, h=2))
    wide = synth.generate(synth.c2_law(8192, 120, 64, seed=22, h=2))
    deep = synth.generate(synth.c3_law(1500, 300, 100, seed=23, h=4))
    return [(synth.generate(synth.c2_law(2000, 300, 200, seed=1, h=3)), 3), (small, 2), (small, 3), (small, 1),
            (deep, 4), (wide, 2), (wide, 1)]


def _noalloc(mh, torch, stream, c, h):
    d_bm = torch.from_numpy(c.bitmaps.view(np.int64)).to("cuda")
    cap = c.Nt
    genes = torch.full((cap * h,), -1, dtype=torch.int32, device="cuda")
    tp = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    fp = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    k, rounds = mh.mh_solve_noalloc(d_bm.data_ptr(), c.G, c.Nt, c.Nn, h, ALPHA, stream.cuda_stream,
                                    genes.data_ptr(), tp.data_ptr(), fp.data_ptr(), cap)
    g = genes.cpu().numpy()[:k * h].reshape(k, h)
    return [(tuple(int(x) for x in g[i]), int(tp[i]), int(fp[i])) for i in range(k)], rounds


def test_noalloc_matches_solve_on_consecutive_calls():
    mh = _lib()
    import torch

    stream = torch.cuda.Stream()
    cohorts = _cohorts()
    refs = []
    for c, h in cohorts:
        with mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) as H:
            refs.append(mh.mh_solve(H, h, ALPHA))
    for call in range(2):  # two calls in a row on each input, interleaved
        for (c, h), ref in zip(cohorts, refs):
            got, rounds = _noalloc(mh, torch, stream, c, h)
            assert got == ref.records(), f"call {call}, G={c.G}, h={h}"
            assert rounds == ref.rounds


def test_noalloc_frontier_overflow_then_correct():
    """A depth-2 frontier beyond 2^17 prefixes: MH_ENOMEM with the limit in the
    message; the shared scratch then still gives mh_solve's results."""
    mh = _lib()
    import torch

    stream = torch.cuda.Stream()
    dense = synth.generate(synth.CohortSpec(G=2000, Nt=300, Nn=60, law=synth.LAW_LOGNORMAL, seed=24, h=3,
                                            ln_mu=float(np.log(0.25)), ln_sigma=0.2, p_lo=0.2, p_hi=0.3))
    with pytest.raises(mh.MHError) as e:
        _noalloc(mh, torch, stream, dense, 3)
    assert e.value.code == mh.MH_ENOMEM and "131072" in str(e.value)
    c = synth.generate(synth.c2_law(900, 190, 70, seed=21, h=3))
    with mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) as H:
        ref = mh.mh_solve(H, 3, ALPHA)
    got, rounds = _noalloc(mh, torch, stream, c, 3)
    assert got == ref.records() and rounds == ref.rounds


def test_noalloc_rejects_sizes_beyond_its_scratch():
    mh = _lib()
    import torch

    d = torch.zeros(9000 * 2, dtype=torch.int64, device="cuda")
    out = torch.zeros(64 * 3, dtype=torch.int32, device="cuda")
    with pytest.raises(mh.MHError) as e:
        mh.mh_solve_noalloc(d.data_ptr(), 9000, 64, 64, 3, ALPHA, 0, out.data_ptr(), out.data_ptr(),
                            out.data_ptr(), 64)
    assert e.value.code == mh.MH_EINVAL and "8192" in str(e.value)
