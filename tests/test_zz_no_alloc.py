"""mh_solve_noalloc: the solve for callers that cannot allocate device memory.

Such callers (code running while another component owns all device memory
through its own pool, plug-ins handed fixed buffers, latency-critical streams
that must not see allocator traffic) get every piece of scratch from one fixed
__device__ array inside the library.  This file runs last so that a failure
here leaves every other test already run.  The entry point is called through
the C ABI and must return exactly what mh_solve returns, on consecutive calls
that reuse the shared scratch array.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _cohorts():
    small = synth.generate(synth.c2_law(900, 190, 70, seed=21, h=2))
    return [(synth.generate(synth.c2_law(2000, 300, 200, seed=1, h=3)), 3), (small, 2), (small, 3)]


def test_noalloc_matches_solve_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_16721_gb300 import mh

    stream = torch.cuda.Stream()
    cohorts = _cohorts()
    refs = []
    for c, h in cohorts:
        with mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) as H:
            refs.append(mh.mh_solve(H, h, (1, 10)))
    for call in range(2):  # two calls in a row on each input, interleaved
        for (c, h), ref in zip(cohorts, refs):
            d_bm = torch.from_numpy(c.bitmaps.view(np.int64)).to("cuda")
            cap = c.Nt
            genes = torch.full((cap * h,), -1, dtype=torch.int32, device="cuda")
            tp = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
            fp = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            k, rounds = mh.mh_solve_noalloc(d_bm.data_ptr(), c.G, c.Nt, c.Nn, h, (1, 10), stream.cuda_stream,
                                            genes.data_ptr(), tp.data_ptr(), fp.data_ptr(), cap)
            g = genes.cpu().numpy()[:k * h].reshape(k, h)
            got = [(tuple(int(x) for x in g[i]), int(tp[i]), int(fp[i])) for i in range(k)]
            assert got == ref.records(), f"call {call}, G={c.G}, h={h}"
            assert rounds == ref.rounds


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_2603_16721_gb300 import mh

    d = torch.zeros(9000 * 2, dtype=torch.int64, device="cuda")
    out = torch.zeros(64 * 3, dtype=torch.int32, device="cuda")
    with pytest.raises(mh.MHError) as e:
        mh.mh_solve_noalloc(d.data_ptr(), 9000, 64, 64, 3, (1, 10), 0, out.data_ptr(), out.data_ptr(),
                            out.data_ptr(), 64)
    assert e.value.code == mh.MH_EINVAL and "8192" in str(e.value)
