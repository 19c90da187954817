"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: bit-exact -- the same ordered combinations with the same TP / FP, and the
same per-round visited / pruned counters of the P-DFS tree (all integer work).
"""
import hashlib
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from golden_io import GOLDEN, load_hand_cases
from test_oracle_pins import _random_cohort

pytestmark = pytest.mark.gpu

HAND = load_hand_cases()


@pytest.fixture(scope="module")
def mh():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_16721_gb300 import mh as m
    return m


def _gpu(mh, bm, G, Nt, Nn, h, alpha=(1, 10), **kw):
    with mh.mh_create(bm, G, Nt, Nn) as H:
        return mh.mh_solve_ex(H, h, alpha, **kw)


def _same(gpu, ref, counters=True):
    assert gpu.records() == ref.records()
    if counters:
        assert gpu.visited.shape == ref.visited.shape
        assert np.array_equal(gpu.visited, ref.visited)
        assert np.array_equal(gpu.pruned, ref.pruned)


@pytest.mark.parametrize("case", HAND, ids=[c.name for c in HAND])
def test_hand_cases(mh, case):
    bm = case.bitmaps()
    for prune in (mh.MH_PRUNE_PAPER, mh.MH_PRUNE_OFF):
        for mode in (mh.MH_MODE_PERSISTENT, mh.MH_MODE_LAUNCHES):
            got = _gpu(mh, bm, case.G, case.Nt, case.Nn, case.h, case.alpha, prune=prune, mode=mode)
            assert got.records() == case.expect
            ref = oracle.pdfs(bm, case.G, case.Nt, case.Nn, case.h, case.alpha, prune=prune == mh.MH_PRUNE_PAPER)
            _same(got, ref)


@pytest.mark.parametrize("seed", range(60))
def test_random_small(mh, seed):
    rng = np.random.default_rng(500 + seed)
    h = int(rng.integers(1, 6))
    G = int(rng.integers(max(h, 2), 90 if h <= 3 else 40))
    Nt = int(rng.integers(1, 300))
    Nn = int(rng.integers(0, 200))
    bm, _, _ = _random_cohort(rng, G, Nt, Nn, rng.uniform(0.02, 0.4), rng.uniform(0.0, 0.3))
    alpha = [(1, 10), (1, 1), (3, 7), (0, 1), (7, 2)][seed % 5]
    ref = oracle.pdfs(bm, G, Nt, Nn, h, alpha)
    _same(_gpu(mh, bm, G, Nt, Nn, h, alpha), ref)
    _same(_gpu(mh, bm, G, Nt, Nn, h, alpha, mode=mh.MH_MODE_LAUNCHES), ref)
    if G <= 40 and h <= 3:
        _same(_gpu(mh, bm, G, Nt, Nn, h, alpha, prune=mh.MH_PRUNE_OFF),
              oracle.pdfs(bm, G, Nt, Nn, h, alpha, prune=False))


@pytest.mark.parametrize("h", [5, 6, 7, 8, 9])
def test_deep_h(mh, h):
    """Deep searches (prefixes of up to 8 genes, three tuple words in the key)."""
    rng = np.random.default_rng(h)
    G, Nt, Nn = 26, 150, 40
    bm, _, _ = _random_cohort(rng, G, Nt, Nn, 0.55, 0.3)
    _same(_gpu(mh, bm, G, Nt, Nn, h), oracle.pdfs(bm, G, Nt, Nn, h))


def test_ragged_sizes_and_wide_rows(mh):
    """Rows of 1..32 words, genes across several 64-gene column words and a ragged tail."""
    rng = np.random.default_rng(9)
    for Nt, Nn, G in [(1, 0, 3), (64, 64, 65), (65, 1, 129), (2048, 2048, 200), (1000, 700, 333)]:
        bm, _, _ = _random_cohort(rng, G, Nt, Nn, 4.0 / max(G, 1) + 0.01, 0.02)
        for h in (1, 2, 3):
            _same(_gpu(mh, bm, G, Nt, Nn, h), oracle.pdfs(bm, G, Nt, Nn, h))


def test_c1_full_matches_bruteforce(mh):
    c = synth.generate(synth.c1())
    brute = oracle.bruteforce(c.bitmaps, c.G, c.Nt, c.Nn, 2)
    got = _gpu(mh, c.bitmaps, c.G, c.Nt, c.Nn, 2)
    assert got.records() == brute.records()
    _same(got, oracle.pdfs(c.bitmaps, c.G, c.Nt, c.Nn, 2))
    # planted pairs are found first
    assert {tuple(sorted(p)) for p in c.planted.tolist()} == {got.records()[0][0], got.records()[1][0]}


def _golden(name, spec, h):
    path = os.path.join(GOLDEN, f"{name}.json")
    c = synth.generate(spec)
    if os.path.exists(path):
        g = json.load(open(path))
        if g["cohort_sha256"] == hashlib.sha256(c.bitmaps.tobytes()).hexdigest():
            recs = [(tuple(x[0]), x[1], x[2]) for x in g["records"]]
            return c, recs, np.array(g["visited"], dtype=np.uint64), np.array(g["pruned"], dtype=np.uint64)
    sol = oracle.pdfs(c.bitmaps, c.G, c.Nt, c.Nn, h)  # generator differs here: recompute the oracle
    return c, sol.records(), sol.visited, sol.pruned


def test_c2_full_solve_matches_oracle(mh):
    """The benchmark workload (h=3, G=5,000, Nt=500, Nn=300), whole greedy solve."""
    c, recs, vis, pru = _golden("c2_pdfs", synth.c2(), 3)
    for mode in (mh.MH_MODE_PERSISTENT, mh.MH_MODE_LAUNCHES):
        got = _gpu(mh, c.bitmaps, c.G, c.Nt, c.Nn, 3, mode=mode)
        assert got.mode == mode
        assert got.records() == recs
        assert np.array_equal(got.visited, vis) and np.array_equal(got.pruned, pru)


def test_c2_exhaustive_first_round_counts(mh):
    """Pruning off on the benchmark cohort: round 1 visits C(G-h+l, l) nodes per depth and picks
    the same combination as the pruned search."""
    c = synth.generate(synth.c2())
    off = _gpu(mh, c.bitmaps, c.G, c.Nt, c.Nn, 3, prune=mh.MH_PRUNE_OFF, max_rounds=1)
    on = _gpu(mh, c.bitmaps, c.G, c.Nt, c.Nn, 3, max_rounds=1)
    assert [int(v) for v in off.visited[0]] == [math.comb(c.G - 3 + l, l) for l in (1, 2, 3)]
    assert off.records() == on.records()
    assert int(off.visited[0, 2] - off.pruned[0, 2]) == int(on.visited[0, 2] - on.pruned[0, 2])


def _replay_checks(c, got, h):
    """Sampled outputs checked one by one: TP / FP of every selection against the mask U
    left by the previous selections; invariants of the whole solve."""
    U = oracle.full_tumor_mask(c.Nt)
    covered = 0
    for genes, tp, fp in got.records():
        rtp, rfp = oracle.cover_counts(c.bitmaps, c.G, c.Nt, c.Nn, np.array([genes], dtype=np.int32), U)
        assert (tp, fp) == (int(rtp[0]), int(rfp[0])) and tp >= 1
        covered += tp
        y = U.copy()
        for g in genes:
            y &= c.bitmaps[g, :c.Wt]
        U &= ~y
    T = np.unpackbits(np.ascontiguousarray(c.bitmaps[:, :c.Wt]).view(np.uint8), bitorder="little",
                      axis=1)[:, :c.Nt]
    assert covered == int((T.sum(axis=0) >= h).sum())  # final cover = coverable tumors
    assert len(set(got.records())) == got.k


def test_c3_law_small_matches_oracle(mh):
    spec = synth.c3_law(600, 800, 400, seed=12, h=4)
    c = synth.generate(spec)
    _same(_gpu(mh, c.bitmaps, c.G, c.Nt, c.Nn, 4), oracle.pdfs(c.bitmaps, c.G, c.Nt, c.Nn, 4))


def test_create_device_and_repeat_are_identical(mh):
    torch = pytest.importorskip("torch")
    c = synth.generate(synth.c2_law(1500, 300, 200, seed=3, h=3))
    ref = oracle.pdfs(c.bitmaps, c.G, c.Nt, c.Nn, 3)
    dev = torch.from_numpy(c.bitmaps.view(np.int64)).cuda()
    s = torch.cuda.Stream()
    with mh.mh_create_device(dev.data_ptr(), c.G, c.Nt, c.Nn, s.cuda_stream) as H:
        a = mh.mh_solve(H, 3)
        b = mh.mh_solve(H, 3)
    _same(a, ref)
    _same(b, ref)


def test_invalid_inputs_rejected(mh):
    bm = np.zeros((3, 2), dtype=np.uint64)
    bm[0, 0] = np.uint64(1) << np.uint64(40)  # tumor bit 40 with Nt = 10: padding set
    with pytest.raises(mh.MHError) as e:
        mh.mh_create(bm, 3, 10, 10)
    assert e.value.code == mh.MH_EINVAL
    ok = np.zeros((3, 2), dtype=np.uint64)
    with mh.mh_create(ok, 3, 10, 10) as H:
        for h, a in [(0, (1, 10)), (10, (1, 10)), (2, (1, 0)), (2, (-1, 3))]:
            with pytest.raises(mh.MHError) as e:
                mh.mh_solve(H, h, a)
            assert e.value.code == mh.MH_EINVAL


def test_frontier_growth_on_overflow(mh, monkeypatch):
    """Frontiers sized only by growth from small initial regions (16 records per
    shard): the first rounds overflow them, the host grows them and reruns the
    round; results and counters are unchanged."""
    monkeypatch.setenv("MH_FRONTIER_PRESIZE", "0")
    monkeypatch.setenv("MH_FRONTIER_MIN_RECORDS", "16")
    c = synth.generate(synth.c2_law(1500, 300, 200, seed=4, h=4))
    ref = oracle.pdfs(c.bitmaps, c.G, c.Nt, c.Nn, 4)
    for mode in (mh.MH_MODE_PERSISTENT, mh.MH_MODE_LAUNCHES):
        got = _gpu(mh, c.bitmaps, c.G, c.Nt, c.Nn, 4, mode=mode)
        _same(got, ref)
        if mode == mh.MH_MODE_PERSISTENT:
            assert got.kernel_launches > 2   # init + at least one relaunch after an overflow
    handles = [mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) for _ in range(2)]
    try:
        for r in mh.mh_solve_batch(handles, [4, 4], blocks=[8, 8]):
            _same(r, ref)
    finally:
        for H in handles:
            H.close()
