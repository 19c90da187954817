"""Error paths with failures made on the host (nothing faults, traps or hangs the
GPU): an injected device-allocation failure in create, solve and served admission
returns MH_ENOMEM and leaves the library usable; an injected timeout report returns
MH_ETIMEOUT and the handle's next solve is correct; cancelled served requests end
with MH_ECANCELED while the others complete; a large request completes while a
stream of small ones keeps the server busy (aging)."""
import threading
import time

import numpy as np
import pytest

import oracle
import synth
from test_oracle_pins import _random_cohort

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mh():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_16721_gb300 import mh as m
    yield m
    m.mh_set_fault(None)


def _small(seed, G=60, Nt=120, Nn=40, h=3):
    rng = np.random.default_rng(seed)
    bm, _, _ = _random_cohort(rng, G, Nt, Nn, 0.12, 0.05)
    return bm, G, Nt, Nn, h


def test_alloc_failure_in_create_and_solve(mh):
    bm, G, Nt, Nn, h = _small(1)
    ref = oracle.pdfs(bm, G, Nt, Nn, h)
    mh.mh_set_fault("alloc_fail=1")
    with pytest.raises(mh.MHError) as e:
        mh.mh_create(bm, G, Nt, Nn)
    assert e.value.code == mh.MH_ENOMEM and "injected" in str(e.value)
    with mh.mh_create(bm, G, Nt, Nn) as H:
        for k in (1, 3, 6):  # the k-th allocation of the first solve's workspace fails
            mh.mh_set_fault(f"alloc_fail={k}")
            with pytest.raises(mh.MHError) as e:
                mh.mh_solve(H, h)
            assert e.value.code == mh.MH_ENOMEM
        mh.mh_set_fault(None)
        got = mh.mh_solve(H, h)
    assert got.records() == ref.records()
    assert np.array_equal(got.visited, ref.visited) and np.array_equal(got.pruned, ref.pruned)


def test_timeout_report_leaves_handle_usable(mh):
    bm, G, Nt, Nn, h = _small(2)
    ref = oracle.pdfs(bm, G, Nt, Nn, h)
    with mh.mh_create(bm, G, Nt, Nn) as H:
        mh.mh_set_fault("timeout_after=1")
        with pytest.raises(mh.MHError) as e:
            mh.mh_solve(H, h)
        assert e.value.code == mh.MH_ETIMEOUT and "injected" in str(e.value)
        got = mh.mh_solve(H, h)
    assert got.records() == ref.records()


def test_alloc_failure_in_served_admission(mh):
    reqs = [_small(10 + i) for i in range(3)]
    with mh.Server(slots=2) as S:
        mh.mh_set_fault("alloc_fail=1")
        t0 = S.submit(*reqs[0])
        with pytest.raises(mh.MHError) as e:
            S.wait(t0, 60000)
        assert e.value.code == mh.MH_ENOMEM
        mh.mh_set_fault(None)
        ts = [S.submit(*r) for r in reqs[1:]]
        for t, (bm, G, Nt, Nn, h) in zip(ts, reqs[1:]):
            assert S.wait(t, 60000).records() == oracle.pdfs(bm, G, Nt, Nn, h).records()


def test_cancel_queued_and_running(mh):
    big = synth.generate(synth.c3_law(3000, 800, 400, 1000, h=3))
    reqs = [(big.bitmaps, big.G, big.Nt, big.Nn, 3)] + [_small(20 + i) for i in range(5)]
    with mh.Server(slots=1) as S:  # one at a time: the others queue behind the first
        ts = [S.submit(*r) for r in reqs]
        S.cancel(ts[2])   # queued
        S.cancel(ts[0])   # running (or already finished)
        for i, (t, (bm, G, Nt, Nn, h)) in enumerate(zip(ts, reqs)):
            if i == 2:
                with pytest.raises(mh.MHError) as e:
                    S.wait(t, 60000)
                assert e.value.code == mh.MH_ECANCELED
            elif i == 0:
                try:
                    r = S.wait(t, 60000)
                    assert r.records() == oracle.pdfs_mt(bm, G, Nt, Nn, h).records()
                except mh.MHError as e:
                    assert e.code == mh.MH_ECANCELED
            else:
                assert S.wait(t, 60000).records() == oracle.pdfs(bm, G, Nt, Nn, h).records()
        assert S.stats()["queued"] == 0


def test_large_request_completes_under_small_stream(mh):
    """Small requests queued back to back keep the server busy; a large request
    submitted among them must finish long before they drain (it joins a launch
    with them once it has paused for large_wait_ms)."""
    big = synth.generate(synth.c3_law(19000, 800, 400, 1003, h=4))
    smalls = [_small(100 + i, G=120, Nt=300, h=3) for i in range(7)]
    with mh.Server(slots=8, large_wait_ms=20) as S:
        t_start = time.time()
        before = [S.submit(*smalls[i % 7]) for i in range(400)]
        tb = S.submit(big.bitmaps, big.G, big.Nt, big.Nn, 4)
        after = [S.submit(*smalls[i % 7]) for i in range(2000)]
        r = S.wait(tb, 60000)
        t_big = time.time() - t_start
        for t in before + after:
            S.wait(t, 120000)
        t_all = time.time() - t_start
    assert r is not None and r.k > 0
    assert t_big < 0.5 * t_all, (t_big, t_all)
    with mh.mh_create(big.bitmaps, big.G, big.Nt, big.Nn) as H:
        assert r.records() == mh.mh_solve(H, 4).records()
