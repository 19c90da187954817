"""Served runtime: requests that share the GPU through continuous batching get
exactly the result each gets alone."""
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
    return m


def _same(a, b):
    assert a.records() == b.records()
    assert np.array_equal(a.visited, b.visited) and np.array_equal(a.pruned, b.pruned)


def _requests():
    rng = np.random.default_rng(31)
    reqs = []
    for i in range(14):
        h = [2, 3, 4, 1][i % 4]
        G = int(rng.integers(40, 160 if h <= 3 else 60))
        Nt = int(rng.integers(30, 400))
        Nn = int(rng.integers(0, 200))
        bm, _, _ = _random_cohort(rng, G, Nt, Nn, rng.uniform(0.03, 0.25), rng.uniform(0.0, 0.2))
        reqs.append((bm, G, Nt, Nn, h))
    # two larger cohorts drawn like the served workload's members (smaller G)
    for seed, h in ((1000, 3), (1001, 2)):
        c = synth.generate(synth.c3_law(3000, 800, 400, seed, h=h))
        reqs.append((c.bitmaps, c.G, c.Nt, c.Nn, h))
    return reqs


def test_mixed_requests_equal_alone(mh):
    reqs = _requests()
    alone = []
    for bm, G, Nt, Nn, h in reqs:
        with mh.mh_create(bm, G, Nt, Nn) as H:
            alone.append(mh.mh_solve(H, h))
    for (bm, G, Nt, Nn, h), a in list(zip(reqs, alone))[:14]:
        _same(a, oracle.pdfs(bm, G, Nt, Nn, h))
    # the two members drawn like the served workload's: the threaded CPU P-DFS
    # (checked against the oracle on the CPU) finishes them in seconds
    for (bm, G, Nt, Nn, h), a in list(zip(reqs, alone))[14:]:
        _same(a, oracle.pdfs_mt(bm, G, Nt, Nn, h))
    with mh.Server(slots=4) as S:
        tickets = []
        for i, (bm, G, Nt, Nn, h) in enumerate(reqs):  # staggered arrivals join running ones
            tickets.append(S.submit(bm, G, Nt, Nn, h))
            if i % 3 == 0:
                time.sleep(0.002)
        got = [S.wait(t, 60000) for t in tickets]
        assert S.stats()["launches"] >= 1
    for g, a in zip(got, alone):
        assert g is not None
        _same(g, a)
        assert g.solve_ms > 0  # latency from submission


def test_concurrent_submitters_and_polling(mh):
    reqs = _requests()[:8]
    with mh.Server(slots=3) as S:
        out = {}

        def worker(k):
            bm, G, Nt, Nn, h = reqs[k]
            t = S.submit(bm, G, Nt, Nn, h)
            r = None
            while r is None:
                r = S.poll(t)
                time.sleep(0.001)
            out[k] = r

        ths = [threading.Thread(target=worker, args=(k,)) for k in range(len(reqs))]
        for t in ths:
            t.start()
        for t in ths:
            t.join(120)
    for k, (bm, G, Nt, Nn, h) in enumerate(reqs):
        with mh.mh_create(bm, G, Nt, Nn) as H:
            _same(out[k], mh.mh_solve(H, h))


def test_request_above_budget_is_rejected(mh):
    bm, G, Nt, Nn, h = _requests()[0]
    with mh.Server(hbm_budget_bytes=1 << 20, slots=2) as S:
        t = S.submit(bm, G, Nt, Nn, h)
        with pytest.raises(mh.MHError) as e:
            S.wait(t, 30000)
        assert e.value.code == mh.MH_EREJECT
