"""Parity of the search shortcuts with the oracle: subtrees below a node whose tumor
intersection is one sample are counted in closed form, and the TP = 1 leaves they
hold are represented by per-sample champions (the best h-subset of each tumor's
genes valued with TP = 1).  The selections and every per-round counter must stay
those of the oracle's P-DFS (§III-D, Algorithm 2), including where a champion
search gives up (no FP = 0 subset within its budget) and the sample's subtrees
are searched and scored instead.
"""
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


def _same(gpu, ref):
    assert gpu.records() == ref.records()
    assert np.array_equal(gpu.visited, ref.visited)
    assert np.array_equal(gpu.pruned, ref.pruned)


def _both_modes(mh, bm, G, Nt, Nn, h, alpha):
    ref = oracle.pdfs(bm, G, Nt, Nn, h, alpha)
    for mode in (mh.MH_MODE_PERSISTENT, mh.MH_MODE_LAUNCHES):
        with mh.mh_create(bm, G, Nt, Nn) as H:
            _same(mh.mh_solve_ex(H, h, alpha, mode=mode), ref)
    return ref


def _pack(T, N):
    """Packed rows from boolean matrices T (G x Nt) and N (G x Nn)."""
    G, Nt = T.shape
    Nn = N.shape[1]
    Wt, Wn = (Nt + 63) // 64, (Nn + 63) // 64
    bm = np.zeros((G, Wt + Wn), dtype=np.uint64)
    for g in range(G):
        for s in np.flatnonzero(T[g]):
            bm[g, s // 64] |= np.uint64(1) << np.uint64(s % 64)
        for s in np.flatnonzero(N[g]):
            bm[g, Wt + s // 64] |= np.uint64(1) << np.uint64(s % 64)
    return bm


@pytest.mark.parametrize("h", [3, 4])
def test_champion_budget_exceeded_falls_back_to_search(mh, h):
    """A normal sample carrying every gene puts every combination at FP >= 1, so no
    champion search stops early; tumors with 40-70 genes exceed the search budget
    (C(70, 3) and C(40, 4) are above 2^15 subsets) and are searched and scored
    like the rest, the others get an exhaustive champion."""
    rng = np.random.default_rng(40 + h)
    G, Nt, Nn = 80, 90, 12
    T = rng.random((G, Nt)) < 0.04
    heavy = {3: 70, 4: 40}[h]
    for s in (3, 17, 55):
        T[rng.choice(G, heavy, replace=False), s] = True
    N = rng.random((G, Nn)) < 0.05
    N[:, 0] = True
    bm = _pack(T, N)
    _both_modes(mh, bm, G, Nt, Nn, h, (1, 10))


@pytest.mark.parametrize("h,seed", [(2, 0), (3, 1), (4, 2), (5, 3), (4, 4), (3, 5)])
def test_sparse_cohorts_mostly_single_sample(mh, h, seed):
    """Sparse cohorts of the c3 law, scaled down: nearly every node below depth 1
    has one uncovered tumor, so nearly the whole tree is counted in closed form."""
    spec = synth.c3_law(600 if h <= 3 else 250, 160, 90, seed=7000 + seed, h=h, n_plant=2)
    c = synth.generate(spec)
    ref = _both_modes(mh, c.bitmaps, c.G, c.Nt, c.Nn, h, (1, 10))
    assert ref.k > 0


@pytest.mark.parametrize("alpha", [(0, 1), (1, 1), (5, 3)])
def test_alpha_changes_which_leaves_can_win(mh, alpha):
    """With alpha = 0 a TP = 1 leaf scores as much as any leaf with the same FP, and
    champions tie with multi-sample leaves; larger alpha favours wide covers."""
    rng = np.random.default_rng(sum(alpha))
    G, Nt, Nn = 120, 140, 60
    bm, _, _ = _random_cohort(rng, G, Nt, Nn, 0.04, 0.03)
    for h in (2, 3, 4):
        _both_modes(mh, bm, G, Nt, Nn, h, alpha)


def test_batched_and_alone_agree_on_sparse_cohorts(mh):
    """Per-sample champions are computed per cohort inside a batched launch too."""
    specs = [synth.c3_law(500, 120 + 20 * i, 70, seed=7100 + i, h=3 + (i % 2), n_plant=2) for i in range(4)]
    cohorts = [synth.generate(sp) for sp in specs]
    refs = [oracle.pdfs(c.bitmaps, c.G, c.Nt, c.Nn, sp.h) for c, sp in zip(cohorts, specs)]
    handles = [mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) for c in cohorts]
    try:
        for r, ref in zip(mh.mh_solve_batch(handles, [sp.h for sp in specs]), refs):
            _same(r, ref)
    finally:
        for H in handles:
            H.close()
