"""The CUDA path at the full size of the h=4 workload (G=19,000, Nt=800, Nn=400),
where the oracle cannot search a round (C(19000, 4) ~ 5e15 leaves).  Checked one by
one instead, with the oracle's counting routines:

* every selection's TP / FP against the uncovered tumors left by the previous ones;
* sampled optimality: in each of the first rounds no sampled 4-gene set sharing an
  uncovered tumor has a larger key (score, then smaller original tuple; §III-D);
* the depth-1 and depth-2 counters of every round, which follow in closed form from
  the sparsity order (§III-C) and the loop bounds of Algorithm 2;
* the final cover equals the tumors with at least h mutated genes, no combination
  repeats (the closing invariants of Algorithm 1).

And element by element against stored oracle results (tests/golden/, written by
make_oracle_goldens.py from the oracle alone):

* c3_r2: the first two greedy rounds of this workload, every selection and every
  per-depth visited / pruned counter (the oracle needs hours for them);
* c3w_pdfs: the same law at the same sample width (14 tumor words, 7 normal
  words) with G = 5,000, the whole solve (485 selections), every counter.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import synth
from golden_io import GOLDEN
from test_gpu_parity import _replay_checks

pytestmark = pytest.mark.gpu

ALPHA = (1, 10)


@pytest.fixture(scope="module")
def mh():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_16721_gb300 import mh as m
    return m


@pytest.fixture(scope="module")
def c3_solved(mh):
    c = synth.generate(synth.c3())
    with mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) as H:
        got = mh.mh_solve_ex(H, 4, ALPHA)
    return c, got


def _tumor_bits(c):
    return np.unpackbits(np.ascontiguousarray(c.bitmaps[:, :c.Wt]).view(np.uint8), bitorder="little",
                         axis=1)[:, :c.Nt].astype(bool)


def _pack(U):
    """Boolean tumor vector -> LSB-first uint64 words."""
    w = np.packbits(U, bitorder="little")
    return np.concatenate([w, np.zeros((-w.size) % 8, np.uint8)]).view(np.uint64)


def _masks(c, got):
    """U before each round (as a boolean tumor vector)."""
    T = _tumor_bits(c)
    U = np.ones(c.Nt, dtype=bool)
    out = []
    for genes, _, _ in got.records():
        out.append(U.copy())
        U &= ~np.logical_and.reduce(T[list(genes)], axis=0)
    out.append(U.copy())
    return T, out


def test_c3_selections_replay(c3_solved):
    c, got = c3_solved
    assert got.k > 100
    _replay_checks(c, got, 4)


def test_c3_depth1_depth2_counters(c3_solved):
    c, got = c3_solved
    h, G = 4, c.G
    T, masks = _masks(c, got)
    order = oracle.sparsity_order(c.bitmaps, c.G, c.Nt, c.Nn)
    assert sorted(order.tolist()) == list(range(G))
    rows = np.ascontiguousarray(c.bitmaps[order, :c.Wt])   # tumor words in search order
    for r in range(got.rounds):
        nonempty = (rows[:G - h + 1] & _pack(masks[r])).any(axis=1)
        pos = np.nonzero(nonempty)[0]
        assert int(got.visited[r, 0]) == G - h + 1
        assert int(got.pruned[r, 0]) == G - h + 1 - pos.size
        assert int(got.visited[r, 1]) == int((G - h + 1 - pos).sum())


def test_c3_sampled_optimality(c3_solved):
    c, got = c3_solved
    h = 4
    T, masks = _masks(c, got)
    rng = np.random.default_rng(77)
    recs = got.records()
    for r in range(min(25, got.k)):
        U = masks[r]
        tum = np.nonzero(U)[0]
        cand = []
        for s in rng.choice(tum, size=min(400, tum.size), replace=True):
            genes = np.nonzero(T[:, s])[0]
            if genes.size >= h:
                cand.append(np.sort(rng.choice(genes, size=h, replace=False)))
        cand = np.array(cand, dtype=np.int32)
        tp, fp = oracle.cover_counts(c.bitmaps, c.G, c.Nt, c.Nn, cand, _pack(U))
        genes, tp0, fp0 = recs[r]
        s0 = ALPHA[0] * tp0 + ALPHA[1] * (c.Nn - fp0)
        for t, a, b in zip(cand, tp, fp):
            assert a >= 1
            s = ALPHA[0] * int(a) + ALPHA[1] * (c.Nn - int(b))
            assert s < s0 or (s == s0 and tuple(genes) <= tuple(int(x) for x in t))


def _stored(name, spec):
    """Cohort and stored oracle result, or None when this machine's generator drew
    a different cohort (the hash does not match)."""
    path = os.path.join(GOLDEN, f"{name}.json")
    c = synth.generate(spec)
    if not os.path.exists(path):
        return c, None
    g = json.load(open(path))
    if g["cohort_sha256"] != hashlib.sha256(c.bitmaps.tobytes()).hexdigest():
        return c, None
    return c, g


def _same_as_stored(got, g, rounds=None):
    recs = [(tuple(x[0]), x[1], x[2]) for x in g["records"]]
    vis = np.array(g["visited"], dtype=np.uint64)
    pru = np.array(g["pruned"], dtype=np.uint64)
    if rounds is not None:
        recs, vis, pru = recs[:rounds], vis[:rounds], pru[:rounds]
    assert got.records() == recs
    assert got.visited.shape == vis.shape
    assert np.array_equal(got.visited, vis) and np.array_equal(got.pruned, pru)


def test_c3_first_rounds_match_stored_oracle(mh):
    c, g = _stored("c3_r2", synth.c3())
    if g is None:
        pytest.skip("no stored oracle result for this machine's c3 cohort (the oracle needs hours)")
    R = len(g["visited"])
    for mode in (mh.MH_MODE_PERSISTENT, mh.MH_MODE_LAUNCHES):
        with mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) as H:
            got = mh.mh_solve_ex(H, 4, ALPHA, max_rounds=R, mode=mode)
        _same_as_stored(got, g, R)


def test_c3w_whole_solve_matches_stored_oracle(mh):
    spec = synth.c3_law(5000, 800, 400, 3)
    c, g = _stored("c3w_pdfs", spec)
    if g is None:  # recompute with the threaded CPU P-DFS (itself checked against the oracle)
        sol = oracle.pdfs_mt(c.bitmaps, c.G, c.Nt, c.Nn, 4, ALPHA)
        g = {"records": [[list(t), a, b] for t, a, b in sol.records()],
             "visited": sol.visited.astype(int).tolist(), "pruned": sol.pruned.astype(int).tolist()}
    for mode in (mh.MH_MODE_PERSISTENT, mh.MH_MODE_LAUNCHES):
        with mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) as H:
            got = mh.mh_solve_ex(H, 4, ALPHA, mode=mode)
        assert got.mode == mode
        _same_as_stored(got, g)
