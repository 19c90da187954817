"""mh_evaluate (the coverage evaluation of §IV-D) on the GPU against the oracle's
definition: random combinations on random cohorts (ragged sample counts), and the
paper's experiment on the synthetic workloads -- learn on a 75% split of the
samples, evaluate on the training and on the held-out 25%."""
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


def _pack_mask(b):
    w = np.packbits(np.asarray(b, dtype=np.uint8), bitorder="little")
    return np.concatenate([w, np.zeros((-w.size) % 8, np.uint8)]).view(np.uint64)


def _same(got, ref, Nt, Nn):
    assert (got["tc"], got["tt"], got["nc"], got["nt"]) == (ref["tc"], ref["tt"], ref["nc"], ref["nt"])
    assert got["sensitivity"] == pytest.approx(ref["sensitivity"], abs=0) or ref["tt"] == 0
    assert np.array_equal(got["tumor_covered"], _pack_mask(ref["tumor_covered"])[:(Nt + 63) // 64])
    assert np.array_equal(got["normal_covered"], _pack_mask(ref["normal_covered"])[:(Nn + 63) // 64])


@pytest.mark.parametrize("seed", range(12))
def test_random_combinations(mh, seed):
    rng = np.random.default_rng(3000 + seed)
    G, Nt, Nn = int(rng.integers(5, 300)), int(rng.integers(1, 700)), int(rng.integers(0, 300))
    h = int(rng.integers(1, 5))
    bm, _, _ = _random_cohort(rng, G, Nt, Nn, rng.uniform(0.05, 0.6), rng.uniform(0.0, 0.5))
    k = int(rng.integers(0, 40))
    combos = np.sort(np.array([rng.choice(G, size=min(h, G), replace=False) for _ in range(k)],
                              dtype=np.int32).reshape(k, min(h, G)), axis=1)
    with mh.mh_create(bm, G, Nt, Nn) as H:
        got = mh.mh_evaluate(H, combos)
    _same(got, oracle.coverage(bm, G, Nt, Nn, combos), Nt, Nn)


@pytest.mark.parametrize("spec", [synth.c1(), synth.c2(), synth.c3_law(5000, 800, 400, 3)], ids=["c1", "c2", "c3w"])
def test_train_test_split(mh, spec):
    c = synth.generate(spec)
    (tr, nt, nn), (te, mt, mn) = synth.split_samples(c, 0.75, seed=7)
    with mh.mh_create(tr, c.G, nt, nn) as H:
        sol = mh.mh_solve(H, spec.h)
        train = mh.mh_evaluate(H, sol.genes)
    with mh.mh_create(te, c.G, mt, mn) as H:
        test = mh.mh_evaluate(H, sol.genes)
    _same(train, oracle.coverage(tr, c.G, nt, nn, sol.genes), nt, nn)
    _same(test, oracle.coverage(te, c.G, mt, mn, sol.genes), mt, mn)
    assert train["tc"] == int(sol.tp.sum())  # training coverage = the greedy cover


def test_bad_indices_rejected(mh):
    bm = np.zeros((4, 2), dtype=np.uint64)
    with mh.mh_create(bm, 4, 64, 64) as H:
        with pytest.raises(mh.MHError) as e:
            mh.mh_evaluate(H, np.array([[0, 4]], dtype=np.int32))
        assert e.value.code == mh.MH_EINVAL
