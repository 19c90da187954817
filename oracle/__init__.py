"""CPU oracle for the greedy multi-hit weighted set cover with P-DFS.

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package; the solver library never does, and the
two share no code.  ``oracle.c`` holds the arithmetic (plain single-threaded C,
no intrinsics); this module compiles it with gcc and marshals arguments.

Functions (all results use original gene indices, ascending inside a tuple):
  bruteforce(...)      -- Algorithm 1 with step F evaluated by plain enumeration
                          of every h-subset (the definition; §II-B, Eq. 1).
  pdfs(...)            -- Algorithm 2 (P-DFS, §III-D) after the sparsity sort of
                          §III-C, with per-round visited / pruned counters.
  sparsity_order(...)  -- the §III-C gene order (ascending tumor mutation count,
                          ties by original index).
  cover_counts(...)    -- TP / FP of given combinations against a mask U.
  pdfs_mt(...)         -- the same P-DFS on several threads (``pdfs_mt.c``: the
                          depth-1 subtrees handed out by an atomic counter, the
                          paper's master-worker scheme of §III-E on host cores),
                          optionally with the score-bound cut; the multi-core
                          CPU baseline.
  mt_round(...)        -- one round of that search over a given U, optionally on
                          one shard of the depth-1 genes (the per-round unit of a
                          multi-process solve); ``delcols(...)`` applies a winner.

Readings of the paper that these functions fix (each is pinned by a test):
  * F = (alpha T+ + T-) / (Nt + Nn) with T- = Nn - FP, FP the normals that
    carry all genes of the combination (coverage in Eq. 1 needs every gene); with
    alpha = a_num / a_den the integer S = a_num TP + a_den (Nn - FP) orders
    candidates exactly as F does.
  * A combination with TP = 0 is never a candidate (§III-D scores only leaves
    with a non-empty intersection).
  * Ties: the lexicographically smallest ascending tuple of original indices.
  * DelCols removes the covered tumors only; the loop stops when every tumor is
    covered or no combination covers an uncovered tumor.
  * Pruning tests the tumor intersection with the uncovered tumors at every depth.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "pdfs_mt.c")]
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, ENOMEM, ECAP = 0, 1, 3, 8


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` and ``pdfs_mt.c`` into ``oracle/liboracle.so``."""
    newest = max(os.path.getmtime(f) for f in _SRCS)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp] + _SRCS)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_bruteforce.restype = ctypes.c_int
        lib.oracle_bruteforce.argtypes = [_P, _I32, _I32, _I32, _I32, _I64, _I64, _I32, _I32,
                                          _P, _P, _P, _P]
        lib.oracle_pdfs.restype = ctypes.c_int
        lib.oracle_pdfs.argtypes = [_P, _I32, _I32, _I32, _I32, _I64, _I64, _I32, _I32, _I32, _I32,
                                    _P, _P, _P, _P, _I32, _P, _P, _P]
        lib.oracle_sparsity_order.restype = ctypes.c_int
        lib.oracle_sparsity_order.argtypes = [_P, _I32, _I32, _I32, _P]
        lib.oracle_cover_counts.restype = ctypes.c_int
        lib.oracle_cover_counts.argtypes = [_P, _I32, _I32, _I32, _I32, _P, _I32, _P, _P, _P]
        lib.pdfs_mt_round.restype = ctypes.c_int
        lib.pdfs_mt_round.argtypes = [_P, _I32, _I32, _I32, _I32, _I64, _I64, _I32, _P, _P, _I32, _I32, _I32,
                                      _P, _P, _P, _P, _P, _P, _P, _P]
        lib.pdfs_mt_delcols.restype = ctypes.c_int
        lib.pdfs_mt_delcols.argtypes = [_P, _I32, _I32, _I32, _I32, _P, _P]
        lib.pdfs_mt_solve.restype = ctypes.c_int
        lib.pdfs_mt_solve.argtypes = [_P, _I32, _I32, _I32, _I32, _I64, _I64, _I32, _I32, _I32, _I32,
                                      _P, _P, _P, _P, _I32, _P, _P, _P, _P]
        _lib = lib
    return _lib


@dataclass
class Solution:
    """Ordered greedy result: genes[k, h] (original indices), tp[k], fp[k]."""
    genes: np.ndarray
    tp: np.ndarray
    fp: np.ndarray
    visited: np.ndarray = field(default=None)   # [rounds, h] (P-DFS only)
    pruned: np.ndarray = field(default=None)    # [rounds, h]

    @property
    def k(self) -> int:
        return int(self.tp.shape[0])

    def tuples(self):
        return [tuple(int(g) for g in row) for row in self.genes]

    def records(self):
        return [(tuple(int(g) for g in self.genes[i]), int(self.tp[i]), int(self.fp[i]))
                for i in range(self.k)]


def _prep(bitmaps, G, Nt, Nn):
    bm = np.ascontiguousarray(bitmaps, dtype=np.uint64)
    W = (Nt + 63) // 64 + (Nn + 63) // 64
    if bm.size != G * W:
        raise ValueError(f"bitmaps hold {bm.size} words, expected G*W = {G * W}")
    return bm


def _check(rc, what):
    if rc == OK:
        return
    raise ValueError(f"{what} failed with status {rc}")


def bruteforce(bitmaps, G, Nt, Nn, h, alpha=(1, 10), max_rounds=-1) -> Solution:
    bm = _prep(bitmaps, G, Nt, Nn)
    cap = Nt + 1
    genes = np.zeros((cap, h), dtype=np.int32)
    tp = np.zeros(cap, dtype=np.int32)
    fp = np.zeros(cap, dtype=np.int32)
    k = ctypes.c_int32()
    rc = _load().oracle_bruteforce(bm.ctypes.data, G, Nt, Nn, h, alpha[0], alpha[1], max_rounds, cap,
                                   genes.ctypes.data, tp.ctypes.data, fp.ctypes.data, ctypes.byref(k))
    _check(rc, "oracle_bruteforce")
    n = k.value
    return Solution(genes[:n].copy(), tp[:n].copy(), fp[:n].copy())


def pdfs(bitmaps, G, Nt, Nn, h, alpha=(1, 10), prune=True, sort=True, max_rounds=-1) -> Solution:
    bm = _prep(bitmaps, G, Nt, Nn)
    cap = Nt + 1
    genes = np.zeros((cap, h), dtype=np.int32)
    tp = np.zeros(cap, dtype=np.int32)
    fp = np.zeros(cap, dtype=np.int32)
    visited = np.zeros((cap + 1, h), dtype=np.uint64)
    pruned = np.zeros((cap + 1, h), dtype=np.uint64)
    k = ctypes.c_int32()
    rounds = ctypes.c_int32()
    rc = _load().oracle_pdfs(bm.ctypes.data, G, Nt, Nn, h, alpha[0], alpha[1], int(bool(prune)),
                             int(bool(sort)), max_rounds, cap, genes.ctypes.data, tp.ctypes.data,
                             fp.ctypes.data, ctypes.byref(k), cap + 1, visited.ctypes.data,
                             pruned.ctypes.data, ctypes.byref(rounds))
    _check(rc, "oracle_pdfs")
    n, r = k.value, rounds.value
    return Solution(genes[:n].copy(), tp[:n].copy(), fp[:n].copy(), visited[:r].copy(), pruned[:r].copy())


def sparsity_order(bitmaps, G, Nt, Nn) -> np.ndarray:
    bm = _prep(bitmaps, G, Nt, Nn)
    order = np.zeros(max(G, 1), dtype=np.int32)
    _check(_load().oracle_sparsity_order(bm.ctypes.data, G, Nt, Nn, order.ctypes.data),
           "oracle_sparsity_order")
    return order[:G]


def cover_counts(bitmaps, G, Nt, Nn, combos, U=None):
    """TP (against U, default all tumors) and FP of each row of ``combos``."""
    bm = _prep(bitmaps, G, Nt, Nn)
    combos = np.ascontiguousarray(combos, dtype=np.int32)
    n, h = combos.shape
    Wt = (Nt + 63) // 64
    if U is None:
        U = full_tumor_mask(Nt)
    U = np.ascontiguousarray(U, dtype=np.uint64)
    assert U.size == Wt
    tp = np.zeros(n, dtype=np.int32)
    fp = np.zeros(n, dtype=np.int32)
    _check(_load().oracle_cover_counts(bm.ctypes.data, G, Nt, Nn, h, U.ctypes.data, n,
                                       combos.ctypes.data, tp.ctypes.data, fp.ctypes.data),
           "oracle_cover_counts")
    return tp, fp


def full_tumor_mask(Nt: int) -> np.ndarray:
    Wt = (Nt + 63) // 64
    U = np.zeros(max(Wt, 1), dtype=np.uint64)
    for w in range(Wt):
        rem = Nt - 64 * w
        U[w] = np.uint64(0xFFFFFFFFFFFFFFFF) if rem >= 64 else np.uint64((1 << rem) - 1)
    return U[:Wt]


# Pruning modes of the threaded P-DFS.
MT_PRUNE_OFF, MT_PRUNE_PAPER, MT_PRUNE_BOUND = 0, 1, 2


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))


def pdfs_mt(bitmaps, G, Nt, Nn, h, alpha=(1, 10), prune=MT_PRUNE_PAPER, max_rounds=-1, threads=None) -> Solution:
    """Threaded P-DFS (``pdfs_mt.c``); ``Solution.cut`` holds the bound-mode cuts."""
    bm = _prep(bitmaps, G, Nt, Nn)
    threads = default_threads() if threads is None else threads
    cap = Nt + 1
    genes = np.zeros((cap, h), dtype=np.int32)
    tp = np.zeros(cap, dtype=np.int32)
    fp = np.zeros(cap, dtype=np.int32)
    visited = np.zeros((cap + 1, h), dtype=np.uint64)
    pruned = np.zeros((cap + 1, h), dtype=np.uint64)
    cut = np.zeros((cap + 1, h), dtype=np.uint64)
    k = ctypes.c_int32()
    rounds = ctypes.c_int32()
    rc = _load().pdfs_mt_solve(bm.ctypes.data, G, Nt, Nn, h, alpha[0], alpha[1], int(prune), max_rounds,
                               int(threads), cap, genes.ctypes.data, tp.ctypes.data, fp.ctypes.data,
                               ctypes.byref(k), cap + 1, visited.ctypes.data, pruned.ctypes.data,
                               cut.ctypes.data, ctypes.byref(rounds))
    _check(rc, "pdfs_mt_solve")
    n, r = k.value, rounds.value
    sol = Solution(genes[:n].copy(), tp[:n].copy(), fp[:n].copy(), visited[:r].copy(), pruned[:r].copy())
    sol.cut = cut[:r].copy()
    return sol


@dataclass
class RoundResult:
    """One round's search on one shard: best candidate (or none) and counters."""
    have: bool
    score: int
    genes: tuple
    tp: int
    fp: int
    visited: np.ndarray
    pruned: np.ndarray
    cut: np.ndarray


def mt_round(bitmaps, G, Nt, Nn, h, U, alpha=(1, 10), prune=MT_PRUNE_PAPER, order=None, threads=1, shard=0,
             nshards=1) -> RoundResult:
    bm = _prep(bitmaps, G, Nt, Nn)
    order = sparsity_order(bm, G, Nt, Nn) if order is None else np.ascontiguousarray(order, dtype=np.int32)
    U = np.ascontiguousarray(U, dtype=np.uint64)
    have = ctypes.c_int32()
    score = ctypes.c_int64()
    tup = np.zeros(h, dtype=np.int32)
    tp = ctypes.c_int32()
    fp = ctypes.c_int32()
    visited = np.zeros(h, dtype=np.uint64)
    pruned = np.zeros(h, dtype=np.uint64)
    cut = np.zeros(h, dtype=np.uint64)
    rc = _load().pdfs_mt_round(bm.ctypes.data, G, Nt, Nn, h, alpha[0], alpha[1], int(prune), order.ctypes.data,
                               U.ctypes.data, int(threads), int(shard), int(nshards), ctypes.byref(have),
                               ctypes.byref(score), tup.ctypes.data, ctypes.byref(tp), ctypes.byref(fp),
                               visited.ctypes.data, pruned.ctypes.data, cut.ctypes.data)
    _check(rc, "pdfs_mt_round")
    return RoundResult(bool(have.value), int(score.value), tuple(int(x) for x in tup), int(tp.value),
                       int(fp.value), visited, pruned, cut)


def delcols(bitmaps, G, Nt, Nn, genes, U) -> np.ndarray:
    """U with the tumors covered by ``genes`` cleared (Algorithm 1's DelCols)."""
    bm = _prep(bitmaps, G, Nt, Nn)
    out = np.ascontiguousarray(U, dtype=np.uint64).copy()
    t = np.ascontiguousarray(genes, dtype=np.int32)
    _check(_load().pdfs_mt_delcols(bm.ctypes.data, G, Nt, Nn, t.size, t.ctypes.data, out.ctypes.data),
           "pdfs_mt_delcols")
    return out


def coverage(bitmaps, G, Nt, Nn, combos) -> dict:
    """Coverage of combinations on a cohort's samples, the evaluation of §IV-D
    (Tables III and IV): a sample is covered when it carries every gene of at
    least one combination.  TC / NC = covered tumors / normals, TT / NT = all of
    them, sensitivity = TC / TT, specificity = 1 - NC / NT (0.0 for an empty total)."""
    bm = _prep(bitmaps, G, Nt, Nn)
    Wt = (Nt + 63) // 64
    T = np.unpackbits(np.ascontiguousarray(bm[:, :Wt]).view(np.uint8), bitorder="little", axis=1)[:, :Nt] != 0
    N = np.unpackbits(np.ascontiguousarray(bm[:, Wt:]).view(np.uint8), bitorder="little", axis=1)[:, :Nn] != 0
    tcov = np.zeros(Nt, dtype=bool)
    ncov = np.zeros(Nn, dtype=bool)
    for row in np.asarray(combos, dtype=np.int64).reshape(-1, np.asarray(combos).shape[-1] if np.size(combos) else 1):
        if row.size == 0:
            continue
        tcov |= T[row].all(axis=0)
        ncov |= N[row].all(axis=0)
    tc, nc = int(tcov.sum()), int(ncov.sum())
    return {"tc": tc, "tt": Nt, "nc": nc, "nt": Nn, "sensitivity": tc / Nt if Nt else 0.0,
            "specificity": 1.0 - nc / Nn if Nn else 0.0, "tumor_covered": tcov, "normal_covered": ncov}
