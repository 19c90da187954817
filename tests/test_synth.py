"""The synthetic cohort generator: layout, determinism and the stated laws."""
import numpy as np
import pytest

import synth


def _unpack(c):
    bits = lambda a: np.unpackbits(a.view(np.uint8), bitorder="little", axis=1)
    T = bits(np.ascontiguousarray(c.bitmaps[:, :c.Wt]))
    N = bits(np.ascontiguousarray(c.bitmaps[:, c.Wt:]))
    return T, N


@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_layout_and_determinism(name):
    spec = synth.COHORTS[name]()
    a = synth.generate(spec)
    b = synth.generate(spec)
    assert np.array_equal(a.bitmaps, b.bitmaps)
    assert a.bitmaps.shape == (spec.G, a.Wt + a.Wn)
    T, N = _unpack(a)
    assert not T[:, spec.Nt:].any() and not N[:, spec.Nn:].any()  # zero padding
    other = synth.generate(synth.CohortSpec(**{**spec.__dict__, "seed": spec.seed + 17}))
    assert not np.array_equal(a.bitmaps, other.bitmaps)


@pytest.mark.parametrize("name,mean,tol", [("c2", 0.008, 0.0015), ("c3", 0.003, 0.0006)])
def test_mean_density(name, mean, tol):
    c = synth.generate(synth.COHORTS[name]())
    T, N = _unpack(c)
    T = T[:, :c.Nt]
    N = N[:, :c.Nn]
    assert abs(T.mean() - mean) < tol
    assert 0.15 < N.mean() / T.mean() < 0.45  # normal rate 0.3x the tumor rate


def test_c3_has_about_50_genes_above_5_percent():
    c = synth.generate(synth.c3())
    T, _ = _unpack(c)
    n = int((T[:, :c.Nt].mean(axis=1) > 0.05).sum())
    assert 30 <= n <= 80


@pytest.mark.parametrize("name,frac", [("c1", (0.2, 0.2)), ("c2", (0.10, 0.15)), ("c3", (0.05, 0.10))])
def test_planted_combinations(name, frac):
    spec = synth.COHORTS[name]()
    c = synth.generate(spec)
    T, _ = _unpack(c)
    T = T[:, :c.Nt]
    assert c.planted.shape == (spec.n_plant, spec.plant_h)
    assert len(set(c.planted.ravel().tolist())) == c.planted.size  # distinct genes
    for combo in c.planted:
        covered = np.logical_and.reduce(T[combo], axis=0).sum()
        assert covered >= int(np.floor(frac[0] * spec.Nt + 0.5))


def test_batch_shapes_and_trace():
    specs = synth.batch16()
    assert len(specs) == 16
    assert [s.h for s in specs] == [3] * 12 + [4] * 4
    for s in specs:
        assert 2000 <= s.G <= 19000 and 100 <= s.Nt <= 1000 and 50 <= s.Nn <= 500
    gaps, hs = synth.trace()
    assert gaps.shape == (200,) and set(np.unique(hs).tolist()) <= {2, 3, 4}
    assert 0.1 < gaps.mean() < 0.3
    assert np.array_equal(synth.trace()[1], hs)


def test_stream_is_reproducible_and_mixed():
    a = synth.stream(0, 1000)
    assert np.array_equal(a, synth.stream(0, 1000))
    assert not np.array_equal(a, synth.stream(1, 1000))
    bits = np.unpackbits(a.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.01
