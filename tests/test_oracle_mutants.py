"""The oracle's pins must catch plausible mistakes.

Each mutant below plants one mistake in a temporary copy of ``oracle/oracle.c``
(on the CPU), compiles it, and runs a compact version of the pin suite against it
(hand-derived cohorts, brute force vs P-DFS, invariants, closed-form counters).
The test passes when every mutant is caught and the unmodified source passes.
"""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from golden_io import load_hand_cases
from test_oracle_pins import _check_invariants, _random_cohort

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "score_drops_fp": [("a_den * (int64_t)(Nn - FP)", "a_den * (int64_t)(Nn)"),
                       ("st->a_den * (int64_t)(st->Nn - FP)", "st->a_den * (int64_t)(st->Nn)")],
    "score_fp_sign": [("a_den * (int64_t)(Nn - FP)", "a_den * (int64_t)(Nn + FP)"),
                      ("st->a_den * (int64_t)(st->Nn - FP)", "st->a_den * (int64_t)(st->Nn + FP)")],
    "alpha_on_wrong_term": [("a_num * (int64_t)TP + a_den * (int64_t)(Nn - FP)",
                             "a_den * (int64_t)TP + a_num * (int64_t)(Nn - FP)"),
                            ("st->a_num * (int64_t)TP + st->a_den * (int64_t)(st->Nn - FP)",
                             "st->a_den * (int64_t)TP + st->a_num * (int64_t)(st->Nn - FP)")],
    "tie_break_reversed": [("tuple_less(t, st->best, h)", "tuple_less(st->best, t, h)"),
                           ("if (!have || S > best_s)", "if (!have || S >= best_s)")],
    "depth_bound_off_by_one": [("const int last = st->G - h + level - 1;",
                                "const int last = st->G - h + level - 2;")],
    "no_delcols": [("for (int w = 0; w < Wt; ++w) U[w] &= ~ybest[w]; /* DelCols on the tumors */", ""),
                   ("for (int w = 0; w < st.Wt; ++w) U[w] &= ~ybest[w];", "")],
    "normals_read_tumor_words": [("for (int w = 0; w < Wn; ++w) n[w] &= row[Wt + w];",
                                  "for (int w = 0; w < Wn; ++w) n[w] &= row[w];"),
                                 ("for (int w = 0; w < Wn; ++w) nc[w] = np[w] & row[Wt + w];",
                                  "for (int w = 0; w < Wn; ++w) nc[w] = np[w] & row[w];")],
    "tp_zero_is_candidate": [("if (TP > 0) {", "if (TP >= 0) {"),
                             ("if (empty) continue; /* TP = 0: not a candidate */", "")],
    "cover_is_union": [("for (int w = 0; w < Wt; ++w) y[w] &= row[w];",
                        "for (int w = 0; w < Wt; ++w) y[w] = (i ? y[w] | (row[w] & U[w]) : y[w] & row[w]);")],
    "last_word_dropped": [("for (int i = 0; i < n; ++i) c += popcount64(w[i]);",
                           "for (int i = 0; i + 1 < n; ++i) c += popcount64(w[i]);")],
    "prune_on_normals": [("const int empty = !any_words(yc, Wt);", "const int empty = !any_words(nc, Wn);")],
}


def _compile(src_text, out_dir, name):
    c = os.path.join(out_dir, f"{name}.c")
    so = os.path.join(out_dir, f"{name}.so")
    with open(c, "w") as f:
        f.write(src_text)
    # the threaded P-DFS is linked in unchanged: the binding loads its symbols too
    mt = os.path.join(os.path.dirname(oracle.__file__), "pdfs_mt.c")
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", so, c, mt])
    return so


def _pin_suite():
    """Compact pin suite; returns the name of the first failing pin, or None."""
    try:
        for case in load_hand_cases():
            bm = case.bitmaps()
            if oracle.bruteforce(bm, case.G, case.Nt, case.Nn, case.h, case.alpha).records() != case.expect:
                return f"hand:{case.name}:brute"
            if oracle.pdfs(bm, case.G, case.Nt, case.Nn, case.h, case.alpha).records() != case.expect:
                return f"hand:{case.name}:pdfs"
        for seed in range(25):
            rng = np.random.default_rng(seed)
            h = int(rng.integers(1, 4))
            G = int(rng.integers(max(h, 2), 16))
            Nt = int(rng.integers(1, 131))
            Nn = int(rng.integers(1, 80))
            bm, T, N = _random_cohort(rng, G, Nt, Nn, rng.uniform(0.1, 0.5), rng.uniform(0.0, 0.4))
            b = oracle.bruteforce(bm, G, Nt, Nn, h)
            try:
                _check_invariants(b, bm, T, N, h, Nn, (1, 10))
            except AssertionError:
                return f"invariants:{seed}"
            p = oracle.pdfs(bm, G, Nt, Nn, h, prune=False)
            if p.records() != b.records():
                return f"brute_vs_pdfs:{seed}"
            for r in range(p.visited.shape[0]):
                if [int(v) for v in p.visited[r]] != [math.comb(G - h + l, l) for l in range(1, h + 1)]:
                    return f"closed_form:{seed}"
    except (AssertionError, ValueError) as e:  # a crash of the pins also counts as caught
        return f"error:{e}"
    return None


def _with_lib(so):
    saved = oracle._lib
    oracle._lib = None
    real_build = oracle.build
    oracle.build = lambda force=False: so
    try:
        oracle._load()
        return _pin_suite()
    finally:
        oracle._lib = saved
        oracle.build = real_build


def test_unmodified_oracle_passes_compact_suite():
    assert _pin_suite() is None


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    src = open(SRC).read()
    mutated = src
    for old, new in MUTANTS[name]:
        assert old in mutated, f"mutation anchor not found: {old!r}"
        mutated = mutated.replace(old, new)
    with tempfile.TemporaryDirectory() as d:
        so = _compile(mutated, d, f"mut_{name}")
        caught = _with_lib(so)
    assert caught is not None, f"mutant {name} survived the pins"
