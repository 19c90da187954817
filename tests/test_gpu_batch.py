"""Batched solve: every cohort of one persistent launch gets exactly the result it
gets alone (selections, TP/FP and per-round counters), for fixed and autotuned
block splits."""
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


def _same(a, b):
    assert a.records() == b.records()
    assert np.array_equal(a.visited, b.visited) and np.array_equal(a.pruned, b.pruned)


def _mixed_cohorts():
    rng = np.random.default_rng(77)
    out = []
    for i, (G, Nt, Nn, h) in enumerate([(60, 130, 40, 2), (45, 70, 0, 3), (30, 200, 90, 4), (120, 64, 64, 1),
                                        (80, 300, 150, 3), (25, 129, 65, 5)]):
        bm, _, _ = _random_cohort(rng, G, Nt, Nn, rng.uniform(0.05, 0.3), rng.uniform(0.0, 0.2))
        out.append((bm, G, Nt, Nn, h))
    return out


def test_batch_equals_alone_and_oracle(mh, tmp_path, monkeypatch):
    monkeypatch.setenv("MH_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    cohorts = _mixed_cohorts()
    handles = [mh.mh_create(bm, G, Nt, Nn) for bm, G, Nt, Nn, h in cohorts]
    hs = [c[4] for c in cohorts]
    alone = [mh.mh_solve(H, h) for H, h in zip(handles, hs)]
    for (bm, G, Nt, Nn, h), a in zip(cohorts, alone):
        _same(a, oracle.pdfs(bm, G, Nt, Nn, h))
    for blocks in ([1] * len(handles), [7, 3, 11, 1, 5, 2], None, None):
        got = mh.mh_solve_batch(handles, hs, blocks=blocks)
        for g, a in zip(got, alone):
            _same(g, a)
    assert (tmp_path / "tune.txt").exists()
    for H in handles:
        H.close()


@pytest.mark.parametrize("choice", ["1000", "2002", "2004", "1", "12", "101.5", "210.75"])
def test_every_batch_schedule_equals_alone(mh, monkeypatch, choice):
    """Each schedule the autotuner can pick -- in turn (1000), groups of 2 and 4
    (2002, 2004), and concurrent launches of each build, work model and split
    exponent (100 * build + 10 * model + gamma) -- gives every cohort the result it
    gets alone."""
    monkeypatch.setenv("MH_BATCH_CHOICE", choice)
    cohorts = _mixed_cohorts()
    handles = [mh.mh_create(bm, G, Nt, Nn) for bm, G, Nt, Nn, h in cohorts]
    hs = [c[4] for c in cohorts]
    alone = [mh.mh_solve(H, h) for H, h in zip(handles, hs)]
    got = mh.mh_solve_batch(handles, hs)
    for g, a in zip(got, alone):
        _same(g, a)
    for H in handles:
        H.close()


def test_batch_of_c2_law_cohorts(mh, tmp_path, monkeypatch):
    """Sixteen cohorts drawn like the batched workload's members, at reduced sizes."""
    monkeypatch.setenv("MH_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    specs = []
    for i, s in enumerate(synth.batch16()):
        specs.append(synth.c2_law(max(300, s.G // 10), max(64, s.Nt // 4), max(32, s.Nn // 4), s.seed, h=s.h))
    cohorts = [synth.generate(sp) for sp in specs]
    handles = [mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) for c in cohorts]
    hs = [sp.h for sp in specs]
    got = mh.mh_solve_batch(handles, hs)
    for c, sp, g in zip(cohorts, specs, got):
        _same(g, oracle.pdfs(c.bitmaps, c.G, c.Nt, c.Nn, sp.h))
    for H in handles:
        H.close()


def test_full_size_batch16_members(mh, tmp_path, monkeypatch):
    """The batched workload at full size in one call: every member equals its solo
    solve, and the two members the CPU finishes in seconds (G = 2,050 and 4,098,
    h = 3) equal the threaded CPU P-DFS (checked against the oracle on the CPU)."""
    monkeypatch.setenv("MH_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    specs = synth.batch16()
    cohorts = [synth.generate(sp) for sp in specs]
    handles = [mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) for c in cohorts]
    try:
        hs = [sp.h for sp in specs]
        got = mh.mh_solve_batch(handles, hs)
        for H, h, g in zip(handles, hs, got):
            _same(g, mh.mh_solve(H, h))
        for i in (3, 1):
            c = cohorts[i]
            _same(got[i], oracle.pdfs_mt(c.bitmaps, c.G, c.Nt, c.Nn, hs[i]))
    finally:
        for H in handles:
            H.close()


def test_batch_rejects_bad_splits(mh):
    bm = np.zeros((4, 2), dtype=np.uint64)
    a = mh.mh_create(bm, 4, 64, 64)
    b = mh.mh_create(bm, 4, 64, 64)
    with pytest.raises(mh.MHError):
        mh.mh_solve_batch([a, b], [2, 2], blocks=[0, 3])
    with pytest.raises(mh.MHError):
        mh.mh_solve_batch([a, a], [2, 2])
    with pytest.raises(mh.MHError):
        mh.mh_solve_batch([a, b], [2, 2], blocks=[10 ** 6, 1])
    a.close()
    b.close()


def test_batch_blocks_numbered_sm_major(mh):
    """A batched launch numbers its blocks SM by SM (teams own whole SMs)."""
    cohorts = _mixed_cohorts()[:3]
    handles = [mh.mh_create(bm, G, Nt, Nn) for bm, G, Nt, Nn, h in cohorts]
    got = mh.mh_solve_batch(handles, [c[4] for c in cohorts], blocks=[8, 8, 8])
    assert all(r.diag[6] == 1 for r in got)
    for H in handles:
        H.close()


def test_batch_start_replays_a_captured_graph(mh, tmp_path, monkeypatch):
    """On a non-default stream the start of a batched solve (every cohort's round
    state and the first cooperative launch) runs from a captured CUDA graph; solving
    the same cohorts again replays it, with the results of solving each alone."""
    import torch
    monkeypatch.setenv("MH_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    monkeypatch.setenv("MH_AUTOTUNE", "0")
    cohorts = _mixed_cohorts()
    stream = torch.cuda.Stream()
    handles = [mh.mh_create(bm, G, Nt, Nn) for bm, G, Nt, Nn, h in cohorts]
    try:
        for H in handles:
            mh.mh_set_stream(H, stream.cuda_stream)
        hs = [h for *_, h in cohorts]
        alone = [mh.mh_solve(H, h) for H, h in zip(handles, hs)]
        for _ in range(3):
            rs = mh.mh_solve_batch(handles, hs)
            for r, a in zip(rs, alone):
                _same(r, a)
                assert r.diag[7] == 1
    finally:
        for H in handles:
            H.close()
