"""The score-bound mode (MH_PRUNE_BOUND): paper pruning plus the cut of every
prefix whose score bound a_num |y| + a_den Nn is below a candidate already found.
It is an addition (the paper uses no branch and bound), so its selections must
be exactly those of the paper's search; its counters depend on when candidates
were found and are only checked against the paper's tree (never more visited
nodes) and for cuts that happened."""
import numpy as np
import pytest

import oracle
import synth
from golden_io import load_hand_cases
from test_gpu_fullsize import _stored
from test_oracle_pins import _random_cohort

pytestmark = pytest.mark.gpu

HAND = load_hand_cases()


@pytest.fixture(scope="module")
def mh():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_16721_gb300 import mh as m
    return m


def _solve(mh, bm, G, Nt, Nn, h, alpha=(1, 10), **kw):
    with mh.mh_create(bm, G, Nt, Nn) as H:
        return mh.mh_solve_ex(H, h, alpha, **kw)


@pytest.mark.parametrize("case", HAND, ids=[c.name for c in HAND])
def test_hand_cases(mh, case):
    bm = case.bitmaps()
    for mode in (mh.MH_MODE_PERSISTENT, mh.MH_MODE_LAUNCHES):
        got = _solve(mh, bm, case.G, case.Nt, case.Nn, case.h, case.alpha, prune=mh.MH_PRUNE_BOUND, mode=mode)
        assert got.records() == case.expect


@pytest.mark.parametrize("seed", range(30))
def test_random_small(mh, seed):
    rng = np.random.default_rng(1500 + seed)
    h = int(rng.integers(1, 6))
    G = int(rng.integers(max(h, 2), 90 if h <= 3 else 40))
    Nt = int(rng.integers(1, 300))
    Nn = int(rng.integers(0, 200))
    bm, _, _ = _random_cohort(rng, G, Nt, Nn, rng.uniform(0.02, 0.4), rng.uniform(0.0, 0.3))
    alpha = [(1, 10), (1, 1), (3, 7), (0, 1), (7, 2)][seed % 5]
    ref = oracle.pdfs(bm, G, Nt, Nn, h, alpha)
    cpu = oracle.pdfs_mt(bm, G, Nt, Nn, h, alpha, prune=oracle.MT_PRUNE_BOUND, threads=2)
    assert cpu.records() == ref.records()
    for mode in (mh.MH_MODE_PERSISTENT, mh.MH_MODE_LAUNCHES):
        got = _solve(mh, bm, G, Nt, Nn, h, alpha, prune=mh.MH_PRUNE_BOUND, mode=mode)
        assert got.records() == ref.records()
        assert got.visited.shape == ref.visited.shape
        assert (got.visited <= ref.visited).all()


@pytest.mark.parametrize("name,spec,h", [("c2_pdfs", synth.c2(), 3), ("c3w_pdfs", synth.c3_law(5000, 800, 400, 3), 4)])
def test_workloads_keep_their_selections(mh, name, spec, h):
    c, g = _stored(name, spec)
    if g is None:
        g = {"records": [[list(t), a, b] for t, a, b in oracle.pdfs_mt(c.bitmaps, c.G, c.Nt, c.Nn, h).records()]}
    recs = [(tuple(x[0]), x[1], x[2]) for x in g["records"]]
    got = _solve(mh, c.bitmaps, c.G, c.Nt, c.Nn, h, prune=mh.MH_PRUNE_BOUND)
    assert got.records() == recs
    assert int(got.cut.sum()) > 0
    if "visited" in g:
        assert int(got.visited.sum()) < int(np.array(g["visited"], dtype=np.uint64).sum())
