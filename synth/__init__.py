"""Seeded synthetic mutation cohorts (inputs only; none of the method's arithmetic).

The paper's cohorts (TCGA somatic mutations, §IV-B) are not available, so these
stand in for them: binary gene x sample matrices with very sparse, heavy-tailed
per-gene rates (a few very frequently mutated genes and a long tail of rare
ones, the profile of §III-A) and a few
planted co-mutated gene combinations.  The generator is plain C
(``cohort_gen.c``), loaded through ctypes, so that cohorts with ~20k genes are
drawn in well under a second.  Both the oracle and the CUDA library take the
layout produced here:

    row g = [ceil(Nt/64) tumor words | ceil(Nn/64) normal words]   (uint64)
    sample s of a block = bit (s % 64) of word (s // 64), LSB first, zero padding.

Named workloads (``COHORTS``):
  c1  h=2, G=1,000, Nt=200, Nn=100, seed 0; per-gene rate
      clip(LogNormal(ln 0.01, 1.0), 0.001, 0.30); normal rate 0.3x;
      two pairs planted in exactly 40 tumors.
  c2  h=3, G=5,000, Nt=500, Nn=300, seed 1; top 20 genes U[0.10, 0.40], the
      rest min(0.10, c r^-0.65) with mean rate 0.008; three triples planted in
      10-15% of tumors.
  c3  h=4, G=19,000, Nt=800, Nn=400, seed 2; min(0.30, c r^-0.65) with mean
      rate 0.003 (about 50 genes above 5%), per-sample burden
      exp(0.7 z - 0.245); four quadruples planted in 5-10% of tumors.
  batch16   16 cohorts, seeds 100-115, G~U[2000,19000], Nt~U[100,1000],
            Nn~U[50,500]; h=3 for the first 12, h=4 for the last 4; c2 law.
  served200 200 requests with c3-law cohorts, seeds 1000-1199; exponential
            arrival gaps of mean 0.2 s; h from {2: .3, 3: .5, 4: .2}; trace
            seed 5000.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cohort_gen.c")
_LIB = os.path.join(_HERE, "libmhgen.so")


def build(force: bool = False) -> str:
    """Compile the generator into ``synth/libmhgen.so`` (gcc, -O2, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("G", ctypes.c_int32), ("Nt", ctypes.c_int32), ("Nn", ctypes.c_int32),
        ("law", ctypes.c_int32),
        ("ln_mu", ctypes.c_double), ("ln_sigma", ctypes.c_double),
        ("p_lo", ctypes.c_double), ("p_hi", ctypes.c_double),
        ("n_top", ctypes.c_int32),
        ("top_lo", ctypes.c_double), ("top_hi", ctypes.c_double), ("beta", ctypes.c_double),
        ("p_cap", ctypes.c_double), ("mean_rate", ctypes.c_double), ("burden_sigma", ctypes.c_double),
        ("normal_ratio", ctypes.c_double),
        ("n_plant", ctypes.c_int32), ("plant_h", ctypes.c_int32),
        ("f_lo", ctypes.c_double), ("f_hi", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.mhgen_generate.restype = ctypes.c_int
        lib.mhgen_generate.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_void_p]
        lib.mhgen_draw_shape.restype = None
        lib.mhgen_draw_shape.argtypes = [ctypes.c_uint64] + [ctypes.c_int32] * 6 + [
            ctypes.POINTER(ctypes.c_int32)] * 3
        lib.mhgen_trace.restype = None
        lib.mhgen_trace.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.mhgen_stream.restype = None
        lib.mhgen_stream.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p]
        _lib = lib
    return _lib


LAW_LOGNORMAL, LAW_POWER_TOP, LAW_POWER_BURDEN = 0, 1, 2


@dataclass(frozen=True)
class CohortSpec:
    """Generator parameters of one cohort (see the module docstring)."""
    G: int
    Nt: int
    Nn: int
    law: int
    seed: int
    h: int = 2                  # hit count the workload is solved with
    ln_mu: float = 0.0
    ln_sigma: float = 0.0
    p_lo: float = 0.0
    p_hi: float = 1.0
    n_top: int = 0
    top_lo: float = 0.0
    top_hi: float = 0.0
    beta: float = 0.65
    p_cap: float = 1.0
    mean_rate: float = 0.0
    burden_sigma: float = 0.0
    normal_ratio: float = 0.3
    n_plant: int = 0
    plant_h: int = 0
    f_lo: float = 0.0
    f_hi: float = 0.0


@dataclass
class Cohort:
    spec: CohortSpec
    bitmaps: np.ndarray      # uint64 [G, Wt + Wn]
    planted: np.ndarray      # int32 [n_plant, plant_h], final row indices

    @property
    def G(self):
        return self.spec.G

    @property
    def Nt(self):
        return self.spec.Nt

    @property
    def Nn(self):
        return self.spec.Nn

    @property
    def Wt(self):
        return (self.spec.Nt + 63) // 64

    @property
    def Wn(self):
        return (self.spec.Nn + 63) // 64


def generate(spec: CohortSpec) -> Cohort:
    lib = _load()
    p = _Params(spec.G, spec.Nt, spec.Nn, spec.law, spec.ln_mu, spec.ln_sigma, spec.p_lo, spec.p_hi,
                spec.n_top, spec.top_lo, spec.top_hi, spec.beta, spec.p_cap, spec.mean_rate,
                spec.burden_sigma, spec.normal_ratio, spec.n_plant, spec.plant_h, spec.f_lo, spec.f_hi,
                spec.seed)
    W = (spec.Nt + 63) // 64 + (spec.Nn + 63) // 64
    bm = np.zeros((spec.G, W), dtype=np.uint64)
    planted = np.zeros((max(spec.n_plant, 0), max(spec.plant_h, 0)), dtype=np.int32)
    rc = lib.mhgen_generate(ctypes.byref(p), bm.ctypes.data, planted.ctypes.data if planted.size else None)
    if rc != 0:
        raise ValueError(f"cohort generator rejected {spec}")
    return Cohort(spec, bm, planted)


def c1(seed: int = 0) -> CohortSpec:
    return CohortSpec(G=1000, Nt=200, Nn=100, law=LAW_LOGNORMAL, seed=seed, h=2,
                      ln_mu=float(np.log(0.01)), ln_sigma=1.0, p_lo=0.001, p_hi=0.30,
                      normal_ratio=0.3, n_plant=2, plant_h=2, f_lo=0.2, f_hi=0.2)


def c2_law(G: int, Nt: int, Nn: int, seed: int, h: int = 3, n_plant: int = 3) -> CohortSpec:
    return CohortSpec(G=G, Nt=Nt, Nn=Nn, law=LAW_POWER_TOP, seed=seed, h=h,
                      n_top=20, top_lo=0.10, top_hi=0.40, beta=0.65, p_cap=0.10, mean_rate=0.008,
                      normal_ratio=0.3, n_plant=n_plant, plant_h=h, f_lo=0.10, f_hi=0.15)


def c2(seed: int = 1) -> CohortSpec:
    return c2_law(5000, 500, 300, seed, h=3)


def c3_law(G: int, Nt: int, Nn: int, seed: int, h: int = 4, n_plant: int = 4) -> CohortSpec:
    return CohortSpec(G=G, Nt=Nt, Nn=Nn, law=LAW_POWER_BURDEN, seed=seed, h=h,
                      beta=0.65, p_cap=0.30, mean_rate=0.003, burden_sigma=0.7,
                      normal_ratio=0.3, n_plant=n_plant, plant_h=h, f_lo=0.05, f_hi=0.10)


def c3(seed: int = 2) -> CohortSpec:
    return c3_law(19000, 800, 400, seed, h=4)


def batch16(first_seed: int = 100, n: int = 16):
    """The batched workload: shapes drawn per cohort seed, h=3 then h=4."""
    lib = _load()
    out = []
    for i in range(n):
        seed = first_seed + i
        G, Nt, Nn = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        lib.mhgen_draw_shape(seed, 2000, 19000, 100, 1000, 50, 500,
                             ctypes.byref(G), ctypes.byref(Nt), ctypes.byref(Nn))
        h = 3 if i < (n * 12) // 16 else 4
        out.append(c2_law(G.value, Nt.value, Nn.value, seed, h=h))
    return out


def trace(seed: int = 5000, n: int = 200, mean_gap: float = 0.2,
          h_values=(2, 3, 4), h_weights=(0.3, 0.5, 0.2)):
    """Arrival gaps (s) and hit counts of the served workload."""
    lib = _load()
    gaps = np.zeros(n, dtype=np.float64)
    hs = np.zeros(n, dtype=np.int32)
    hv = np.asarray(h_values, dtype=np.int32)
    hw = np.asarray(h_weights, dtype=np.float64)
    lib.mhgen_trace(seed, n, mean_gap, len(hv), hv.ctypes.data, hw.ctypes.data, gaps.ctypes.data,
                    hs.ctypes.data)
    return gaps, hs


def served200(first_seed: int = 1000, n: int = 200, trace_seed: int = 5000):
    gaps, hs = trace(trace_seed, n)
    specs = [c3_law(19000, 800, 400, first_seed + i, h=int(hs[i])) for i in range(n)]
    return specs, gaps


def stream(seed: int, n: int) -> np.ndarray:
    """First n outputs of xoshiro256** seeded through splitmix64(seed)."""
    out = np.zeros(n, dtype=np.uint64)
    _load().mhgen_stream(seed, n, out.ctypes.data)
    return out


COHORTS = {"c1": c1, "c2": c2, "c3": c3}


def split_samples(c: Cohort, train_frac: float = 0.75, seed: int = 7):
    """A random train / test split of a cohort's samples (the 75% / 25% split of
    §IV-B and §IV-D), tumors and normals each: (train bitmaps, Nt, Nn), (test
    bitmaps, Nt, Nn).  The order comes from sorting xoshiro256** outputs seeded by
    `seed` (tumors) and `seed + 1` (normals); every gene keeps its row."""
    def order(n, sd):
        return np.argsort(stream(sd, n), kind="stable") if n else np.zeros(0, dtype=np.int64)

    Wt, Wn = c.Wt, c.Wn
    T = np.unpackbits(np.ascontiguousarray(c.bitmaps[:, :Wt]).view(np.uint8), bitorder="little", axis=1)[:, :c.Nt]
    N = np.unpackbits(np.ascontiguousarray(c.bitmaps[:, Wt:]).view(np.uint8), bitorder="little", axis=1)[:, :c.Nn]
    pt, pn = order(c.Nt, seed), order(c.Nn, seed + 1)
    kt, kn = int(round(train_frac * c.Nt)), int(round(train_frac * c.Nn))

    def pack(Tm, Nm):
        nt, nn = Tm.shape[1], Nm.shape[1]
        wt, wn = (nt + 63) // 64, (nn + 63) // 64
        out = np.zeros((c.G, wt + wn), dtype=np.uint64)
        if nt:
            b = np.packbits(Tm.astype(np.uint8), bitorder="little", axis=1)
            b = np.concatenate([b, np.zeros((c.G, 8 * wt - b.shape[1]), np.uint8)], axis=1)
            out[:, :wt] = np.ascontiguousarray(b).view(np.uint64)
        if nn:
            b = np.packbits(Nm.astype(np.uint8), bitorder="little", axis=1)
            b = np.concatenate([b, np.zeros((c.G, 8 * wn - b.shape[1]), np.uint8)], axis=1)
            out[:, wt:] = np.ascontiguousarray(b).view(np.uint64)
        return out, nt, nn

    train = pack(T[:, np.sort(pt[:kt])], N[:, np.sort(pn[:kn])])
    test = pack(T[:, np.sort(pt[kt:])], N[:, np.sort(pn[kn:])])
    return train, test
