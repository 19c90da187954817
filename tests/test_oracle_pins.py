"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* hand-derived answers on hand-built cohorts (tests/golden/hand_cases.txt);
* Table I of the paper (C(20000, h)) and the closed form C(G-h+l, l) for the
  number of depth-l nodes of the exhaustive search;
* special cases that reduce to the textbook greedy set cover (no normals);
* invariants of the greedy loop (final cover = tumors with >= h mutated genes,
  disjoint TP sets, pruning and sorting never change the result, the bound on
  scored leaves);
* brute force on tiny random cohorts, compared with the separate P-DFS.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from golden_io import GOLDEN, load_hand_cases

CASES = load_hand_cases()


def _solve_all_ways(bm, G, Nt, Nn, h, alpha):
    out = {"brute": oracle.bruteforce(bm, G, Nt, Nn, h, alpha)}
    for prune in (True, False):
        for sort in (True, False):
            out[f"pdfs_prune{int(prune)}_sort{int(sort)}"] = oracle.pdfs(bm, G, Nt, Nn, h, alpha,
                                                                         prune=prune, sort=sort)
    return out


@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_hand_cases(case):
    bm = case.bitmaps()
    for how, sol in _solve_all_ways(bm, case.G, case.Nt, case.Nn, case.h, case.alpha).items():
        assert sol.records() == case.expect, how


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_binomials.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                h, mant, exp = line.split()
                rows.append((int(h), mant, int(exp)))
    return rows


def _truncate3(n: int):
    s = str(n)
    return f"{s[0]}.{s[1:3]}", len(s) - 1


@pytest.mark.parametrize("h,mant,exp", _table1())
def test_table1_closed_form(h, mant, exp):
    assert _truncate3(math.comb(20000, h)) == (mant, exp)


def test_table1_h2_enumerated_by_oracle():
    """The exhaustive h=2 search over 20,000 genes visits Table I's 1.99e8 leaves."""
    G = 20000
    bm = np.ones((G, 1), dtype=np.uint64)  # one tumor, mutated in every gene, no normals
    sol = oracle.pdfs(bm, G, 1, 0, 2, (1, 10), prune=False)
    assert sol.visited.shape[0] == 1
    assert int(sol.visited[0, 1]) == math.comb(G, 2) == 199_990_000
    assert _truncate3(int(sol.visited[0, 1])) == ("1.99", 8)
    assert int(sol.visited[0, 0]) == G - 1
    assert sol.records() == [((0, 1), 1, 0)]


def _random_cohort(rng, G, Nt, Nn, dens_t, dens_n):
    Wt, Wn = (Nt + 63) // 64, (Nn + 63) // 64
    T = rng.random((G, Nt)) < dens_t
    N = rng.random((G, Nn)) < dens_n
    return pack(T, N), T, N


def pack(T, N):
    G, Nt = T.shape
    Nn = N.shape[1]
    Wt, Wn = (Nt + 63) // 64, (Nn + 63) // 64
    bm = np.zeros((G, Wt + Wn), dtype=np.uint64)
    for g in range(G):
        for s in np.flatnonzero(T[g]):
            bm[g, s // 64] |= np.uint64(1 << int(s % 64))
        for s in np.flatnonzero(N[g]):
            bm[g, Wt + s // 64] |= np.uint64(1 << int(s % 64))
    return bm


@pytest.mark.parametrize("h,shape", [(None, (12, 70, 9, 0.30, 0.15)), (2, (24, 130, 70, 0.12, 0.05)),
                                     (3, (20, 100, 40, 0.25, 0.10)), (4, (16, 66, 20, 0.40, 0.20))])
def test_counters_closed_form_exhaustive(h, shape):
    """With pruning off, every round visits C(G-h+l, l) nodes at depth l (Algorithm 2 loop bounds)."""
    G, Nt, Nn, dt, dn = shape
    rng = np.random.default_rng(7)
    bm, _, _ = _random_cohort(rng, G, Nt, Nn, dt, dn)
    for hh in ([1, 2, 3] if h is None else [h]):
        sol = oracle.pdfs(bm, G, Nt, Nn, hh, prune=False)
        expect = [math.comb(G - hh + l, l) for l in range(1, hh + 1)]
        assert sol.visited.shape[0] >= 1
        for r in range(sol.visited.shape[0]):
            assert [int(v) for v in sol.visited[r]] == expect


def test_no_empty_branch_means_full_enumeration():
    """§III-D: if no branch ever empties, P-DFS visits all C(G, h) leaves."""
    G, Nt, h = 14, 3, 3
    bm = np.full((G, 1), 0b111, dtype=np.uint64)
    sol = oracle.pdfs(bm, G, Nt, 0, h, prune=True)
    assert [int(v) for v in sol.visited[0]] == [math.comb(G - h + l, l) for l in range(1, h + 1)]
    assert int(sol.pruned[0].sum()) == 0


def _textbook_greedy_cover(sets, universe):
    """Greedy set cover: repeatedly take the set covering most uncovered elements
    (first in list order on ties) until nothing more can be covered."""
    uncovered = set(universe)
    chosen = []
    while uncovered:
        best, gain = None, 0
        for i, s in enumerate(sets):
            gi = len(s & uncovered)
            if gi > gain:
                best, gain = i, gi
        if best is None:
            break
        chosen.append((best, gain))
        uncovered -= sets[best]
    return chosen


@pytest.mark.parametrize("seed", range(40))
def test_no_normals_is_textbook_greedy_cover(seed):
    """With Nn = 0 the score is a_num * TP: the classic greedy set cover over the
    covers of all h-subsets (enumerated here with itertools and Python sets)."""
    rng = np.random.default_rng(1000 + seed)
    h = int(rng.integers(1, 4))
    G = int(rng.integers(h, 13))
    Nt = int(rng.integers(1, 140))
    T = rng.random((G, Nt)) < rng.uniform(0.1, 0.6)
    bm = pack(T, np.zeros((G, 0), dtype=bool))
    combos = list(itertools.combinations(range(G), h))
    covers = [set(np.flatnonzero(np.logical_and.reduce(T[list(c)], axis=0)).tolist()) for c in combos]
    expect = [(combos[i], gain, 0) for i, gain in _textbook_greedy_cover(covers, range(Nt))]
    alpha = (int(rng.integers(1, 5)), int(rng.integers(1, 20)))
    assert oracle.bruteforce(bm, G, Nt, 0, h, alpha).records() == expect
    assert oracle.pdfs(bm, G, Nt, 0, h, alpha).records() == expect


def _coverable(T, h):
    return set(np.flatnonzero(T.sum(axis=0) >= h).tolist())


def _check_invariants(sol, bm, T, N, h, Nn, alpha):
    G, Nt = T.shape
    covered = set()
    U = set(range(Nt))
    for r, (genes, tp, fp) in enumerate(sol.records()):
        assert list(genes) == sorted(set(genes)) and len(genes) == h
        cover_t = set(np.flatnonzero(np.logical_and.reduce(T[list(genes)], axis=0)).tolist())
        cover_n = np.logical_and.reduce(N[list(genes)], axis=0).sum() if Nn else 0
        assert tp == len(cover_t & U) and tp >= 1
        assert fp == cover_n
        assert not (cover_t & U & covered)
        covered |= cover_t & U
        U -= cover_t
    tuples = [g for g, _, _ in sol.records()]
    assert len(tuples) == len(set(tuples))
    assert sum(tp for _, tp, _ in sol.records()) == len(covered)
    # the loop only ends when no combination covers an uncovered tumor
    assert covered == _coverable(T, h)


@pytest.mark.parametrize("seed", range(120))
def test_bruteforce_equals_pdfs_and_invariants(seed):
    rng = np.random.default_rng(seed)
    h = int(rng.integers(1, 5))
    G = int(rng.integers(max(h, 2), 22 if h < 4 else 17))
    Nt = int(rng.integers(1, 131))
    Nn = int(rng.integers(0, 80))
    bm, T, N = _random_cohort(rng, G, Nt, Nn, rng.uniform(0.05, 0.5), rng.uniform(0.0, 0.4))
    alpha = [(1, 10), (1, 1), (3, 7), (0, 1)][seed % 4]
    brute = oracle.bruteforce(bm, G, Nt, Nn, h, alpha)
    _check_invariants(brute, bm, T, N, h, Nn, alpha)
    for prune in (True, False):
        for sort in (True, False):
            p = oracle.pdfs(bm, G, Nt, Nn, h, alpha, prune=prune, sort=sort)
            assert p.records() == brute.records(), (prune, sort)
    # scored leaves per round are bounded by sum over uncovered tumors of C(m_s, h)
    p = oracle.pdfs(bm, G, Nt, Nn, h, alpha)
    U = np.ones(Nt, dtype=bool)
    for r in range(p.visited.shape[0]):
        m = T[:, U].sum(axis=0)
        bound = sum(math.comb(int(x), h) for x in m)
        scored = int(p.visited[r, h - 1] - p.pruned[r, h - 1])
        assert scored <= bound
        if r < p.k:
            U &= ~np.logical_and.reduce(T[list(p.genes[r])], axis=0)
    # prune on and off see the same leaves with a non-empty intersection
    q = oracle.pdfs(bm, G, Nt, Nn, h, alpha, prune=False)
    assert np.array_equal(p.visited[:, h - 1] - p.pruned[:, h - 1], q.visited[:, h - 1] - q.pruned[:, h - 1])


def test_tie_between_identical_rows():
    """Identical gene rows give equal scores; the smallest original tuple is taken."""
    rng = np.random.default_rng(5)
    T = rng.random((6, 40)) < 0.5
    T[4] = T[1]
    T[5] = T[2]
    N = np.zeros((6, 10), dtype=bool)
    bm = pack(T, N)
    for h in (1, 2, 3):
        a = oracle.bruteforce(bm, 6, 40, 10, h)
        b = oracle.pdfs(bm, 6, 40, 10, h)
        assert a.records() == b.records()
        for genes, _, _ in a.records():
            # a tuple using row 4 (or 5) is never chosen where row 1 (or 2) gives the same cover
            for dup, orig in ((4, 1), (5, 2)):
                if dup in genes and orig not in genes:
                    alt = tuple(sorted(set(genes) - {dup} | {orig}))
                    assert alt > genes


def test_sparsity_order_is_stable_ascending():
    rng = np.random.default_rng(3)
    G, Nt, Nn = 50, 100, 30
    bm, T, _ = _random_cohort(rng, G, Nt, Nn, 0.1, 0.1)
    T[7] = T[3]
    bm = pack(T, np.zeros((G, Nn), dtype=bool))
    order = oracle.sparsity_order(bm, G, Nt, Nn)
    counts = T.sum(axis=1)
    expect = sorted(range(G), key=lambda g: (counts[g], g))
    assert order.tolist() == expect


def test_cover_counts_matches_sets():
    rng = np.random.default_rng(11)
    G, Nt, Nn = 30, 150, 90
    bm, T, N = _random_cohort(rng, G, Nt, Nn, 0.4, 0.4)
    combos = np.array([sorted(rng.choice(G, 3, replace=False)) for _ in range(50)], dtype=np.int32)
    Umask = rng.random(Nt) < 0.7
    U = pack(Umask[None, :], np.zeros((1, 0), dtype=bool))[0]
    tp, fp = oracle.cover_counts(bm, G, Nt, Nn, combos, U)
    for i, c in enumerate(combos):
        assert tp[i] == int((np.logical_and.reduce(T[c], axis=0) & Umask).sum())
        assert fp[i] == int(np.logical_and.reduce(N[c], axis=0).sum())


def test_invalid_arguments_rejected():
    bm = np.zeros((3, 2), dtype=np.uint64)
    for args in [(3, 64, 64, 0), (3, 64, 64, 10), (-1, 64, 64, 2)]:
        with pytest.raises(ValueError):
            oracle.pdfs(bm if args[0] >= 0 else bm[:0], *args)
    with pytest.raises(ValueError):
        oracle.bruteforce(bm, 3, 64, 64, 2, alpha=(1, 0))
