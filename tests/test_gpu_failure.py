"""Failure detection without a GPU fault: a barrier wait that nothing can complete
ends by its bound with MH_ETIMEOUT, and the context stays usable afterwards."""
import time

import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mh():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_16721_gb300 import mh as m
    return m


def test_bounded_wait_times_out_and_context_survives(mh):
    t0 = time.perf_counter()
    assert mh.mh_check_bounded_wait() == mh.MH_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    c = synth.generate(synth.c2_law(400, 130, 70, seed=9, h=3))
    with mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) as H:
        got = mh.mh_solve(H, 3)
    assert got.records() == oracle.pdfs(c.bitmaps, c.G, c.Nt, c.Nn, 3).records()
