"""The threaded CPU P-DFS (oracle/pdfs_mt.c) against the single-threaded oracle.

It is the multi-core CPU baseline and the CPU side of the multi-process round
protocol, so it must give exactly what the pinned oracle gives:

* the same selections and the same per-round, per-depth counters as oracle_pdfs
  on random cohorts, with 1, 3 and 8 threads, pruning on and off (and the same
  selections as the brute-force definition);
* the score-bound mode (cut a prefix whose bound a_num |y| + a_den Nn is below
  the best score found, strictly) never changes the selections, and never visits
  more nodes than paper pruning;
* a round split into shards of the depth-1 genes: the largest shard key is the
  unsharded winner, and the shards' counters sum to the unsharded counters;
* the c1 and c2 workloads against their stored oracle results.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from golden_io import GOLDEN
from test_oracle_pins import _random_cohort


def _random(seed):
    rng = np.random.default_rng(900 + seed)
    h = int(rng.integers(1, 5))
    G = int(rng.integers(max(h, 2), 40 if h <= 3 else 24))
    Nt = int(rng.integers(1, 200))
    Nn = int(rng.integers(0, 100))
    bm, _, _ = _random_cohort(rng, G, Nt, Nn, rng.uniform(0.03, 0.45), rng.uniform(0.0, 0.3))
    alpha = [(1, 10), (1, 1), (3, 7), (0, 1), (7, 2)][seed % 5]
    return bm, G, Nt, Nn, h, alpha


@pytest.mark.parametrize("seed", range(40))
def test_threads_match_oracle(seed):
    bm, G, Nt, Nn, h, alpha = _random(seed)
    ref = oracle.pdfs(bm, G, Nt, Nn, h, alpha)
    assert oracle.bruteforce(bm, G, Nt, Nn, h, alpha).records() == ref.records()
    for threads in (1, 3, 8):
        got = oracle.pdfs_mt(bm, G, Nt, Nn, h, alpha, threads=threads)
        assert got.records() == ref.records()
        assert np.array_equal(got.visited, ref.visited) and np.array_equal(got.pruned, ref.pruned)
        assert not got.cut.any()
    if G <= 24:
        off = oracle.pdfs(bm, G, Nt, Nn, h, alpha, prune=False)
        got = oracle.pdfs_mt(bm, G, Nt, Nn, h, alpha, prune=oracle.MT_PRUNE_OFF, threads=4)
        assert got.records() == off.records()
        assert np.array_equal(got.visited, off.visited) and np.array_equal(got.pruned, off.pruned)


@pytest.mark.parametrize("seed", range(40))
def test_bound_mode_keeps_selections(seed):
    bm, G, Nt, Nn, h, alpha = _random(seed)
    ref = oracle.pdfs(bm, G, Nt, Nn, h, alpha)
    for threads in (1, 4):
        got = oracle.pdfs_mt(bm, G, Nt, Nn, h, alpha, prune=oracle.MT_PRUNE_BOUND, threads=threads)
        assert got.records() == ref.records()
        assert got.visited.shape == ref.visited.shape
        assert (got.visited <= ref.visited).all()


def test_bound_mode_cuts_on_a_planted_cohort():
    c = synth.generate(synth.c2_law(600, 200, 100, seed=31, h=3))
    ref = oracle.pdfs(c.bitmaps, c.G, c.Nt, c.Nn, 3)
    got = oracle.pdfs_mt(c.bitmaps, c.G, c.Nt, c.Nn, 3, prune=oracle.MT_PRUNE_BOUND, threads=1)
    assert got.records() == ref.records()
    assert got.cut.sum() > 0 and got.visited.sum() < ref.visited.sum()


def _key(r):
    return (r.score, tuple(-g for g in r.genes))


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("nshards", [2, 3])
def test_shards_merge_to_unsharded_round(seed, nshards):
    bm, G, Nt, Nn, h, alpha = _random(seed)
    U = oracle.full_tumor_mask(Nt)
    order = oracle.sparsity_order(bm, G, Nt, Nn)
    for _ in range(4):  # the first rounds of the greedy loop
        whole = oracle.mt_round(bm, G, Nt, Nn, h, U, alpha, order=order, threads=2)
        parts = [oracle.mt_round(bm, G, Nt, Nn, h, U, alpha, order=order, threads=2, shard=i, nshards=nshards)
                 for i in range(nshards)]
        assert np.array_equal(sum(p.visited for p in parts), whole.visited)
        assert np.array_equal(sum(p.pruned for p in parts), whole.pruned)
        live = [p for p in parts if p.have]
        assert bool(live) == whole.have
        if not whole.have:
            break
        best = max(live, key=_key)
        assert (best.score, best.genes, best.tp, best.fp) == (whole.score, whole.genes, whole.tp, whole.fp)
        U = oracle.delcols(bm, G, Nt, Nn, whole.genes, U)


@pytest.mark.parametrize("name,h", [("c1_pdfs", 2), ("c2_pdfs", 3)])
def test_workloads_match_stored_oracle(name, h):
    with open(os.path.join(GOLDEN, f"{name}.json")) as f:
        g = json.load(f)
    spec = synth.c1() if name == "c1_pdfs" else synth.c2()
    c = synth.generate(spec)
    if name == "c2_pdfs":  # the whole c2 solve is tens of CPU-seconds: its first rounds
        got = oracle.pdfs_mt(c.bitmaps, c.G, c.Nt, c.Nn, h, tuple(g["alpha"]), max_rounds=3)
    else:
        got = oracle.pdfs_mt(c.bitmaps, c.G, c.Nt, c.Nn, h, tuple(g["alpha"]))
    n = got.k
    assert [[list(t), a, b] for t, a, b in got.records()] == g["records"][:n]
    assert got.visited.astype(int).tolist() == g["visited"][:n]
    assert got.pruned.astype(int).tolist() == g["pruned"][:n]
