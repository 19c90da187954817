"""The two facts the GPU search relies on to skip work, checked on the CPU against
brute force and the oracle.

1. Below a search node whose tumor intersection is one sample, the subtree of
   Algorithm 2 (§III-D) is fixed by that sample's genes after the node's last gene:
   its per-depth visited / surviving counts follow a one-pass recurrence over them
   (f_1(b) = [b <= hi(d+1)], f_k(b) = [b <= hi(d+k)] * sum of f_{k-1} over earlier
   genes, hi(e) = G - h + e - 1; a surviving node ending at b has hi(e+1) - b
   children).
2. In every greedy round (Algorithm 1), the argmax over all candidate leaves equals
   the larger of (a) the best leaf carried by two or more uncovered tumors and (b)
   the best per-sample champion of an uncovered tumor, where a champion is the best
   h-subset of that tumor's genes valued with TP = 1.  Keys compare by score, then
   by the smaller tuple of original indices.
"""
import itertools

import numpy as np
import pytest

import oracle
from test_oracle_pins import _random_cohort


# ---- 1. single-sample subtrees -------------------------------------------------

def _subtree_brute(G, h, d, g, genes):
    """Visited / surviving nodes per depth below a depth-d node with y = {s}, by the
    loops of Algorithm 2 (children g' in (last, hi(depth)], pruned when s lacks g')."""
    vis, alive = [0] * (h + 1), [0] * (h + 1)

    def rec(depth, last):
        if depth == h:
            return
        hi = G - h + depth  # 0-based bound of depth + 1
        for c in range(last + 1, hi + 1):
            vis[depth + 1] += 1
            if c in genes:
                alive[depth + 1] += 1
                rec(depth + 1, c)

    rec(d, g)
    return vis, alive


def _subtree_recurrence(G, h, d, g, genes):
    K, hi0 = h - d, G - h + d - 1
    S, av, vi = [0] * (K + 1), [0] * (K + 1), [0] * (K + 1)
    vi[1] = hi0 + 1 - g
    for b in sorted(x for x in genes if x > g):
        for k in range(K, 0, -1):
            if b > hi0 + k:
                continue
            f = 1 if k == 1 else S[k - 1]
            av[k] += f
            if k < K:
                vi[k + 1] += f * (hi0 + k + 1 - b)
                S[k] += f
    vis, alive = [0] * (h + 1), [0] * (h + 1)
    for k in range(1, K + 1):
        vis[d + k], alive[d + k] = vi[k], av[k]
    return vis, alive


def test_single_sample_subtree_recurrence_matches_algorithm_2():
    rng = np.random.default_rng(11)
    for _ in range(1500):
        G = int(rng.integers(3, 36))
        h = int(rng.integers(2, min(7, G) + 1))
        d = int(rng.integers(1, h))
        g = int(rng.integers(d - 1, G - h + d))  # a valid last gene of a depth-d node
        genes = set(int(x) for x in rng.choice(G, int(rng.integers(0, G + 1)), replace=False))
        genes.add(g)
        assert _subtree_recurrence(G, h, d, g, genes) == _subtree_brute(G, h, d, g, genes)


def test_leaf_parent_closed_form():
    """d = h - 1: G - 1 - g leaves visited, the genes of s after g surviving."""
    rng = np.random.default_rng(12)
    for _ in range(500):
        G = int(rng.integers(3, 40))
        h = int(rng.integers(2, min(6, G) + 1))
        g = int(rng.integers(h - 2, G - 1))
        genes = set(int(x) for x in rng.choice(G, int(rng.integers(0, G + 1)), replace=False)) | {g}
        vis, alive = _subtree_brute(G, h, h - 1, g, genes)
        assert vis[h] == G - 1 - g and alive[h] == sum(1 for x in genes if x > g)


# ---- 2. per-sample champions ---------------------------------------------------

def _better(a, b):
    """Larger score wins, then the lexicographically smaller tuple."""
    if b is None:
        return True
    return a[0] > b[0] or (a[0] == b[0] and a[1] < b[1])


@pytest.mark.parametrize("seed", range(40))
def test_round_argmax_is_best_of_multi_sample_leaves_and_champions(seed):
    rng = np.random.default_rng(300 + seed)
    h = int(rng.integers(2, 4))
    G, Nt, Nn = int(rng.integers(h + 2, 13)), int(rng.integers(4, 40)), int(rng.integers(0, 16))
    bm, T, N = _random_cohort(rng, G, Nt, Nn, rng.uniform(0.2, 0.6), rng.uniform(0.0, 0.4))
    a_num, a_den = [(1, 10), (0, 1), (1, 1), (3, 2)][seed % 4]
    ref = oracle.bruteforce(bm, G, Nt, Nn, h, (a_num, a_den))
    U = np.ones(Nt, dtype=bool)
    tumor_sets = [set(np.flatnonzero(T[g])) for g in range(G)]
    normal_sets = [set(np.flatnonzero(N[g])) for g in range(G)]
    for rnd, (tup, tp, fp) in enumerate(ref.records()):
        best = best_multi = None
        for gam in itertools.combinations(range(G), h):
            y = set.intersection(*(tumor_sets[g] for g in gam)) & set(np.flatnonzero(U))
            if not y:
                continue
            n = len(set.intersection(*(normal_sets[g] for g in gam))) if Nn else 0
            key = (a_num * len(y) + a_den * (Nn - n), gam)
            if _better(key, best):
                best = key
            if len(y) >= 2 and _better(key, best_multi):
                best_multi = key
        assert best[1] == tup, "the brute-force argmax is the oracle's selection"
        champ_best = None
        for s in np.flatnonzero(U):
            genes_s = [g for g in range(G) if T[g, s]]
            for gam in itertools.combinations(genes_s, h):
                n = len(set.intersection(*(normal_sets[g] for g in gam))) if Nn else 0
                key = (a_num * 1 + a_den * (Nn - n), gam)
                if _better(key, champ_best):
                    champ_best = key
        combined = best_multi
        if champ_best is not None and _better(champ_best, combined):
            combined = champ_best
        assert combined[0] == best[0] and combined[1] == best[1], f"round {rnd}"
        # DelCols: remove the covered tumors
        cov = set.intersection(*(tumor_sets[g] for g in tup))
        for s in cov:
            U[s] = False
