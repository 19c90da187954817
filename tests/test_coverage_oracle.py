"""The coverage evaluation of §IV-D (oracle.coverage) against what the paper and
the definition fix: every TC / TT / NC / NT row printed in Tables III and IV gives
the printed sensitivity and specificity when a cohort is built with exactly that
coverage; hand-built overlapping combinations; the greedy solve covers on its own
training samples exactly the tumors with at least h mutated genes; and the 75/25
split keeps every sample exactly once."""
import os

import numpy as np
import pytest

import oracle
import synth
from golden_io import GOLDEN
from test_oracle_pins import pack


def _rows():
    out = []
    with open(os.path.join(GOLDEN, "coverage_tables.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                t, name, hits, tc, tt, nc, nt, sens, spec = line.split()
                out.append((t, name, int(tc), int(tt), int(nc), int(nt), float(sens), float(spec)))
    return out


@pytest.mark.parametrize("row", _rows(), ids=lambda r: f"{r[0]}-{r[1]}")
def test_printed_rows(row):
    _, _, tc, tt, nc, nt, sens, spec = row
    # two genes; the combination {0, 1} covers exactly the first tc tumors and nc normals,
    # gene 0 alone also carries one more tumor and normal (not covered by the pair)
    T = np.zeros((2, tt), dtype=bool)
    N = np.zeros((2, nt), dtype=bool)
    T[:, :tc] = True
    N[:, :nc] = True
    if tc < tt:
        T[0, tc] = True
    if nc < nt:
        N[0, nc] = True
    cov = oracle.coverage(pack(T, N), 2, tt, nt, [[0, 1]])
    assert (cov["tc"], cov["tt"], cov["nc"], cov["nt"]) == (tc, tt, nc, nt)
    assert round(cov["sensitivity"], 4) == sens and round(cov["specificity"], 4) == spec


def test_hand_overlapping_combinations():
    # tumors 0..5, normals 0..3; combos {0,1} covers tumors 0,1 and normal 0; {1,2} covers tumor 1, 2
    T = np.zeros((3, 6), dtype=bool)
    N = np.zeros((3, 4), dtype=bool)
    T[0, [0, 1, 3]] = T[1, [0, 1, 2]] = T[2, [1, 2, 5]] = True
    N[0, [0, 2]] = N[1, [0, 1]] = N[2, [1]] = True
    cov = oracle.coverage(pack(T, N), 3, 6, 4, [[0, 1], [1, 2]])
    assert cov["tumor_covered"].tolist() == [True, True, True, False, False, False]
    assert cov["normal_covered"].tolist() == [True, True, False, False]
    assert (cov["tc"], cov["nc"]) == (3, 2)
    assert cov["sensitivity"] == 0.5 and cov["specificity"] == 0.5
    assert oracle.coverage(pack(T, N), 3, 6, 4, np.zeros((0, 2), dtype=np.int32))["tc"] == 0


def test_training_coverage_is_every_coverable_tumor():
    c = synth.generate(synth.c2_law(500, 160, 90, seed=17, h=3))
    (tr, nt, nn), (te, mt, mn) = synth.split_samples(c, 0.75, seed=5)
    sol = oracle.pdfs(tr, c.G, nt, nn, 3)
    cov = oracle.coverage(tr, c.G, nt, nn, sol.genes)
    T = np.unpackbits(np.ascontiguousarray(tr[:, :(nt + 63) // 64]).view(np.uint8), bitorder="little",
                      axis=1)[:, :nt]
    assert cov["tc"] == int((T.sum(axis=0) >= 3).sum()) == int(sol.tp.sum())
    test = oracle.coverage(te, c.G, mt, mn, sol.genes)
    assert test["tt"] == mt and 0 <= test["tc"] <= mt


def test_split_keeps_every_sample_once():
    c = synth.generate(synth.c2_law(300, 130, 70, seed=3, h=2))
    (tr, nt, nn), (te, mt, mn) = synth.split_samples(c, 0.75, seed=11)
    assert (nt, mt, nn, mn) == (98, 32, 52, 18)
    # every gene keeps its per-split mutation counts summing to the whole
    whole = oracle.coverage(c.bitmaps, c.G, c.Nt, c.Nn, [[g] for g in range(c.G)])
    a = oracle.coverage(tr, c.G, nt, nn, [[g] for g in range(c.G)])
    b = oracle.coverage(te, c.G, mt, mn, [[g] for g in range(c.G)])
    assert a["tc"] + b["tc"] == whole["tc"] and a["nc"] + b["nc"] == whole["nc"]
    for g in range(0, c.G, 37):
        cg = lambda bm, n1, n2: oracle.coverage(bm, c.G, n1, n2, [[g]])
        assert cg(tr, nt, nn)["tc"] + cg(te, mt, mn)["tc"] == cg(c.bitmaps, c.Nt, c.Nn)["tc"]
