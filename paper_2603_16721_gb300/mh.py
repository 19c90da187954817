"""Python binding of libmh (argument marshalling only; declared in include/mh.h).

Every function here forwards to the C ABI of ``libmh.so``; no step of a solve runs
in Python.  The library must have been built (``__graft_entry__.build()``); if it
cannot be loaded, every call raises ``MHLibraryError`` -- there is no fallback.

Names follow the C ABI: ``mh_create``, ``mh_create_device``, ``mh_set_stream``,
``mh_solve``, ``mh_solve_ex``, ``mh_destroy``, ``mh_last_error``,
``mh_handle_info``.  Results come back as ``Result`` objects holding numpy
copies of the library's arrays (the C result is released immediately).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

MH_OK, MH_EINVAL, MH_ENOMEM, MH_ECUDA, MH_ETIMEOUT, MH_EAGAIN, MH_EREJECT, MH_ECANCELED = range(8)
MH_PRUNE_PAPER, MH_PRUNE_OFF, MH_PRUNE_BOUND = 0, 1, 2
MH_MODE_PERSISTENT, MH_MODE_LAUNCHES = 0, 1
_NAMES = {0: "MH_OK", 1: "MH_EINVAL", 2: "MH_ENOMEM", 3: "MH_ECUDA", 4: "MH_ETIMEOUT", 5: "MH_EAGAIN",
          6: "MH_EREJECT", 7: "MH_ECANCELED"}


class MHLibraryError(RuntimeError):
    """libmh.so is missing or cannot be loaded."""


class MHError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class mh_rational(ctypes.Structure):
    _fields_ = [("num", ctypes.c_int32), ("den", ctypes.c_int32)]


class mh_solve_opts(ctypes.Structure):
    _fields_ = [("h", ctypes.c_int32), ("alpha", mh_rational), ("prune", ctypes.c_int32),
                ("max_rounds", ctypes.c_int32), ("time_kernels", ctypes.c_int32), ("mode", ctypes.c_int32)]


class mh_result(ctypes.Structure):
    _fields_ = [("h", ctypes.c_int32), ("k", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("genes", ctypes.POINTER(ctypes.c_int32)), ("tp", ctypes.POINTER(ctypes.c_int32)),
                ("fp", ctypes.POINTER(ctypes.c_int32)), ("visited", ctypes.POINTER(ctypes.c_uint64)),
                ("pruned", ctypes.POINTER(ctypes.c_uint64)), ("solve_ms", ctypes.c_double),
                ("leaf_ms", ctypes.c_double), ("leaf_launches", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("leaf_words", ctypes.c_uint64),
                ("leaf_prefixes", ctypes.c_uint64), ("leaf_scored", ctypes.c_uint64),
                ("leaf_alu_ops", ctypes.c_uint64), ("leaf_dense", ctypes.c_uint64),
                ("level1_ms", ctypes.c_double), ("expand_ms", ctypes.c_double), ("finalize_ms", ctypes.c_double),
                ("mode", ctypes.c_int32), ("diag", ctypes.c_uint64 * 8), ("kernel_ms", ctypes.c_double),
                ("cut", ctypes.POINTER(ctypes.c_uint64))]


_lib = None
_P = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load():
    """Load libmh.so (built beforehand by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise MHLibraryError(f"{path} is missing: build it with __graft_entry__.build()")
    try:
        lib = ctypes.CDLL(path)
    except OSError as e:
        raise MHLibraryError(f"cannot load {path}: {e}") from e
    lib.mh_create.restype = ctypes.c_int
    lib.mh_create.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_P)]
    lib.mh_create_device.restype = ctypes.c_int
    lib.mh_create_device.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, ctypes.POINTER(_P)]
    lib.mh_set_stream.restype = ctypes.c_int
    lib.mh_set_stream.argtypes = [_P, _P]
    lib.mh_solve.restype = ctypes.c_int
    lib.mh_solve.argtypes = [_P, ctypes.c_int32, mh_rational, ctypes.POINTER(ctypes.POINTER(mh_result))]
    lib.mh_solve_ex.restype = ctypes.c_int
    lib.mh_solve_ex.argtypes = [_P, ctypes.POINTER(mh_solve_opts), ctypes.POINTER(ctypes.POINTER(mh_result))]
    lib.mh_result_free.restype = None
    lib.mh_result_free.argtypes = [ctypes.POINTER(mh_result)]
    lib.mh_destroy.restype = None
    lib.mh_destroy.argtypes = [_P]
    lib.mh_last_error.restype = ctypes.c_char_p
    lib.mh_last_error.argtypes = []
    lib.mh_handle_info.restype = ctypes.c_int
    lib.mh_handle_info.argtypes = [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]
    _lib = lib
    return lib


def mh_check_bounded_wait() -> int:
    """Status of a barrier wait that only its bound can end (MH_ETIMEOUT expected)."""
    lib = load()
    lib.mh_check_bounded_wait.restype = ctypes.c_int
    lib.mh_check_bounded_wait.argtypes = [ctypes.POINTER(ctypes.c_int32)]
    st = ctypes.c_int32(0)
    _check(lib.mh_check_bounded_wait(ctypes.byref(st)))
    return int(st.value)


class mh_round_best(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("have", ctypes.c_int32), ("score", ctypes.c_int64),
                ("genes", ctypes.c_int32 * 9), ("visited", ctypes.c_uint64 * 9), ("pruned", ctypes.c_uint64 * 9)]


class Shard:
    """One rank's share of a split solve (``mh_shard_*``): search a round, commit the
    merged round, read the result.  Closed with ``mh_shard_free``."""

    def __init__(self, handle: "Handle", h: int, alpha=(1, 10), shard: int = 0, nshards: int = 1,
                 prune: int = MH_PRUNE_PAPER):
        lib = load()
        lib.mh_shard_begin.restype = ctypes.c_int
        lib.mh_shard_begin.argtypes = [_P, ctypes.POINTER(mh_solve_opts), ctypes.c_int32, ctypes.c_int32,
                                       ctypes.POINTER(_P)]
        lib.mh_shard_search.restype = ctypes.c_int
        lib.mh_shard_search.argtypes = [_P, ctypes.POINTER(mh_round_best)]
        lib.mh_shard_commit.restype = ctypes.c_int
        lib.mh_shard_commit.argtypes = [_P, ctypes.POINTER(mh_round_best), ctypes.POINTER(ctypes.c_int32)]
        lib.mh_shard_result.restype = ctypes.c_int
        lib.mh_shard_result.argtypes = [_P, ctypes.POINTER(ctypes.POINTER(mh_result))]
        lib.mh_shard_free.restype = None
        lib.mh_shard_free.argtypes = [_P]
        self.h = h
        opts = mh_solve_opts(h=h, alpha=mh_rational(*alpha), prune=prune, mode=MH_MODE_LAUNCHES)
        p = _P()
        _check(lib.mh_shard_begin(handle.ptr, ctypes.byref(opts), shard, nshards, ctypes.byref(p)))
        self.ptr = p

    def search(self) -> dict:
        rb = mh_round_best()
        _check(load().mh_shard_search(self.ptr, ctypes.byref(rb)))
        h = self.h
        return {"done": bool(rb.done), "have": bool(rb.have), "score": int(rb.score),
                "genes": tuple(int(g) for g in rb.genes[:h]),
                "visited": np.array(rb.visited[:h], dtype=np.uint64), "pruned": np.array(rb.pruned[:h], dtype=np.uint64)}

    def commit(self, merged: dict) -> bool:
        rb = mh_round_best()
        rb.have = int(bool(merged["have"]))
        rb.score = int(merged["score"])
        for i, g in enumerate(merged["genes"]):
            rb.genes[i] = int(g)
        for i in range(self.h):
            rb.visited[i] = int(merged["visited"][i])
            rb.pruned[i] = int(merged["pruned"][i])
        done = ctypes.c_int32(0)
        _check(load().mh_shard_commit(self.ptr, ctypes.byref(rb), ctypes.byref(done)))
        return bool(done.value)

    def result(self) -> "Result":
        out = ctypes.POINTER(mh_result)()
        _check(load().mh_shard_result(self.ptr, ctypes.byref(out)))
        return _to_result(out)

    def close(self):
        if self.ptr:
            load().mh_shard_free(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class mh_coverage(ctypes.Structure):
    _fields_ = [("tc", ctypes.c_int32), ("tt", ctypes.c_int32), ("nc", ctypes.c_int32), ("nt", ctypes.c_int32),
                ("sensitivity", ctypes.c_double), ("specificity", ctypes.c_double)]


def mh_evaluate(handle: "Handle", genes) -> dict:
    """Coverage of combinations (rows of original gene indices) on the handle's
    samples: tc, tt, nc, nt, sensitivity, specificity and the covered masks."""
    lib = load()
    lib.mh_evaluate.restype = ctypes.c_int
    lib.mh_evaluate.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(mh_coverage), _P, _P]
    g = np.ascontiguousarray(genes, dtype=np.int32)
    if g.ndim != 2:
        raise ValueError("genes must be a [k, h] array")
    k, h = g.shape
    G, Nt, Nn, _ = mh_handle_info(handle)
    tmask = np.zeros(max(1, (Nt + 63) // 64), dtype=np.uint64)
    nmask = np.zeros(max(1, (Nn + 63) // 64), dtype=np.uint64)
    out = mh_coverage()
    _check(lib.mh_evaluate(handle.ptr, g.ctypes.data if k else None, k, max(h, 1), ctypes.byref(out),
                           tmask.ctypes.data, nmask.ctypes.data))
    return {"tc": out.tc, "tt": out.tt, "nc": out.nc, "nt": out.nt, "sensitivity": out.sensitivity,
            "specificity": out.specificity, "tumor_covered": tmask[:(Nt + 63) // 64],
            "normal_covered": nmask[:(Nn + 63) // 64]}


def mh_set_fault(spec) -> None:
    """Host-side fault injection: "alloc_fail=N", "timeout_after=N" or None / "none"."""
    lib = load()
    lib.mh_set_fault.restype = ctypes.c_int
    lib.mh_set_fault.argtypes = [ctypes.c_char_p]
    _check(lib.mh_set_fault(spec.encode() if spec else None))


def mh_int_peak(op: int = 0):
    """Measured integer throughput of the current GPU: (thread ops/s, kernel ms) of
    op 0 = LOP3, 1 = POPC, 2 = IADD."""
    lib = load()
    lib.mh_int_peak.restype = ctypes.c_int
    lib.mh_int_peak.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    v = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    _check(lib.mh_int_peak(op, ctypes.byref(v), ctypes.byref(ms)))
    return float(v.value), float(ms.value)


def mh_l2_latency() -> float:
    """Time of one dependent L2 load on the current GPU, in ns."""
    lib = load()
    lib.mh_l2_latency.restype = ctypes.c_int
    lib.mh_l2_latency.argtypes = [ctypes.POINTER(ctypes.c_double)]
    v = ctypes.c_double(0.0)
    _check(lib.mh_l2_latency(ctypes.byref(v)))
    return float(v.value)


def mh_last_error() -> str:
    return load().mh_last_error().decode()


def _check(rc):
    if rc != MH_OK:
        raise MHError(rc, mh_last_error())


@dataclass
class Result:
    """A solve's ordered selections plus per-round counters and timings."""
    h: int
    genes: np.ndarray     # [k, h] original indices, ascending per row
    tp: np.ndarray        # [k]
    fp: np.ndarray        # [k]
    visited: np.ndarray   # [rounds, h]
    pruned: np.ndarray    # [rounds, h]
    solve_ms: float
    leaf_ms: float
    leaf_launches: int
    kernel_launches: int
    leaf_words: int
    leaf_prefixes: int
    leaf_scored: int = 0
    leaf_alu_ops: int = 0
    leaf_dense: int = 0
    level1_ms: float = 0.0
    expand_ms: float = 0.0
    finalize_ms: float = 0.0
    mode: int = 0
    diag: tuple = ()
    kernel_ms: float = 0.0
    cut: np.ndarray = None    # [rounds, h] prefixes cut by the score bound (MH_PRUNE_BOUND)

    @property
    def k(self) -> int:
        return int(self.tp.shape[0])

    @property
    def rounds(self) -> int:
        return int(self.visited.shape[0])

    def records(self):
        return [(tuple(int(g) for g in self.genes[i]), int(self.tp[i]), int(self.fp[i])) for i in range(self.k)]


def _to_result(p) -> Result:
    r = p.contents
    k, h, rounds = r.k, r.h, r.rounds
    arr = lambda ptr, n, dt: np.ctypeslib.as_array(ptr, shape=(n,)).astype(dt, copy=True) if n else np.zeros(0, dt)
    out = Result(h=h,
                 genes=arr(r.genes, k * h, np.int32).reshape(k, h),
                 tp=arr(r.tp, k, np.int32), fp=arr(r.fp, k, np.int32),
                 visited=arr(r.visited, rounds * h, np.uint64).reshape(rounds, h),
                 pruned=arr(r.pruned, rounds * h, np.uint64).reshape(rounds, h),
                 solve_ms=float(r.solve_ms), leaf_ms=float(r.leaf_ms), leaf_launches=int(r.leaf_launches),
                 kernel_launches=int(r.kernel_launches), leaf_words=int(r.leaf_words),
                 leaf_prefixes=int(r.leaf_prefixes), leaf_scored=int(r.leaf_scored),
                 leaf_alu_ops=int(r.leaf_alu_ops), leaf_dense=int(r.leaf_dense),
                 level1_ms=float(r.level1_ms), expand_ms=float(r.expand_ms), finalize_ms=float(r.finalize_ms),
                 mode=int(r.mode), diag=tuple(int(x) for x in r.diag), kernel_ms=float(r.kernel_ms),
                 cut=(arr(r.cut, rounds * h, np.uint64).reshape(rounds, h) if r.cut
                      else np.zeros((rounds, h), np.uint64)))
    load().mh_result_free(p)
    return out


class Handle:
    """Owns an ``mh_handle*``; destroyed with ``mh_destroy`` when closed or collected."""

    def __init__(self, ptr):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            load().mh_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def mh_create(bitmaps: np.ndarray, G: int, Nt: int, Nn: int) -> Handle:
    """Handle from packed rows in host memory (uint64, G x (Wt + Wn))."""
    bm = np.ascontiguousarray(bitmaps, dtype=np.uint64)
    W = (Nt + 63) // 64 + (Nn + 63) // 64
    if bm.size != G * W:
        raise MHError(MH_EINVAL, f"bitmaps hold {bm.size} words, expected {G * W}")
    out = _P()
    _check(load().mh_create(bm.ctypes.data, G, Nt, Nn, ctypes.byref(out)))
    return Handle(out)


def mh_create_device(d_bitmaps_ptr: int, G: int, Nt: int, Nn: int, stream: int = 0) -> Handle:
    """Handle from packed rows in device memory (a raw device pointer, e.g.
    ``tensor.data_ptr()``) and a raw ``cudaStream_t`` (e.g. ``torch_stream.cuda_stream``)."""
    out = _P()
    _check(load().mh_create_device(_P(d_bitmaps_ptr), G, Nt, Nn, _P(stream or None), ctypes.byref(out)))
    return Handle(out)


def mh_set_stream(handle: Handle, stream: int = 0) -> None:
    _check(load().mh_set_stream(handle.ptr, _P(stream or None)))


def mh_solve(handle: Handle, h: int, alpha=(1, 10)) -> Result:
    p = ctypes.POINTER(mh_result)()
    _check(load().mh_solve(handle.ptr, h, mh_rational(*alpha), ctypes.byref(p)))
    return _to_result(p)


def mh_solve_ex(handle: Handle, h: int, alpha=(1, 10), prune: int = MH_PRUNE_PAPER, max_rounds: int = 0,
                time_kernels: bool = False, mode: int = MH_MODE_PERSISTENT) -> Result:
    o = mh_solve_opts(h, mh_rational(*alpha), prune, max_rounds, int(bool(time_kernels)), mode)
    p = ctypes.POINTER(mh_result)()
    _check(load().mh_solve_ex(handle.ptr, ctypes.byref(o), ctypes.byref(p)))
    return _to_result(p)


def mh_destroy(handle: Handle) -> None:
    handle.close()


def mh_handle_info(handle: Handle):
    G, Nt, Nn, b = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(load().mh_handle_info(handle.ptr, ctypes.byref(G), ctypes.byref(Nt), ctypes.byref(Nn), ctypes.byref(b)))
    return G.value, Nt.value, Nn.value, b.value


def mh_solve_noalloc(d_bitmaps_ptr: int, G: int, Nt: int, Nn: int, h: int, alpha, stream: int,
                     d_genes_ptr: int, d_tp_ptr: int, d_fp_ptr: int, capacity: int):
    """Allocation-free greedy solve (see include/mh.h): device input rows, device
    output buffers (int32: capacity*h genes, capacity TP, capacity FP).  Returns
    (k, rounds)."""
    lib = load()
    if not hasattr(lib, "_noalloc_typed"):
        lib.mh_solve_noalloc.restype = ctypes.c_int
        lib.mh_solve_noalloc.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         mh_rational, _P, _P, _P, _P, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
        lib._noalloc_typed = True
    k, rounds = ctypes.c_int32(), ctypes.c_int32()
    _check(lib.mh_solve_noalloc(_P(d_bitmaps_ptr), G, Nt, Nn, h, mh_rational(*alpha), _P(stream or None),
                                _P(d_genes_ptr), _P(d_tp_ptr), _P(d_fp_ptr), capacity, ctypes.byref(k),
                                ctypes.byref(rounds)))
    return k.value, rounds.value


def mh_solve_batch(handles, hs, alphas=None, blocks=None, prune: int = MH_PRUNE_PAPER, max_rounds: int = 0):
    """Solve several cohorts in one persistent launch (see include/mh.h).
    handles: list of Handle; hs: hit count per cohort; alphas: (num, den) per
    cohort (default 1/10); blocks: block split per cohort or None (autotuned)."""
    lib = load()
    if not hasattr(lib, "_batch_typed"):
        lib.mh_solve_batch.restype = ctypes.c_int
        lib.mh_solve_batch.argtypes = [ctypes.POINTER(_P), ctypes.POINTER(mh_solve_opts), ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.POINTER(mh_result))]
        lib._batch_typed = True
    n = len(handles)
    alphas = alphas or [(1, 10)] * n
    ptrs = (_P * n)(*[h.ptr for h in handles])
    opts = (mh_solve_opts * n)(*[mh_solve_opts(int(hs[i]), mh_rational(*alphas[i]), prune, max_rounds, 0,
                                               MH_MODE_PERSISTENT) for i in range(n)])
    b = (ctypes.c_int32 * n)(*blocks) if blocks is not None else None
    outs = (ctypes.POINTER(mh_result) * n)()
    _check(lib.mh_solve_batch(ptrs, opts, n, b, outs))
    return [_to_result(outs[i]) for i in range(n)]


class mh_server_opts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("slots", ctypes.c_int32), ("large_slots", ctypes.c_int32),
                ("large_wait_ms", ctypes.c_int32)]


class Server:
    """Served runtime (continuous batching): mh_server_create / mh_submit /
    mh_poll / mh_wait / mh_server_destroy."""

    def __init__(self, hbm_budget_bytes: int = 0, slots: int = 0, large_slots: int = 0, large_wait_ms: int = 0):
        lib = load()
        if not hasattr(lib, "_server_typed"):
            lib.mh_server_create.restype = ctypes.c_int
            lib.mh_server_create.argtypes = [ctypes.POINTER(mh_server_opts), ctypes.POINTER(_P)]
            lib.mh_submit.restype = ctypes.c_int
            lib.mh_submit.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      mh_rational, ctypes.POINTER(ctypes.c_uint64)]
            lib.mh_poll.restype = ctypes.c_int
            lib.mh_poll.argtypes = [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.POINTER(mh_result))]
            lib.mh_wait.restype = ctypes.c_int
            lib.mh_wait.argtypes = [_P, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(ctypes.POINTER(mh_result))]
            lib.mh_server_stats.restype = ctypes.c_int
            lib.mh_server_stats.argtypes = [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]
            lib.mh_server_destroy.restype = None
            lib.mh_server_destroy.argtypes = [_P]
            lib.mh_cancel.restype = ctypes.c_int
            lib.mh_cancel.argtypes = [_P, ctypes.c_uint64]
            lib._server_typed = True
        self.ptr = _P()
        o = mh_server_opts(hbm_budget_bytes, slots, large_slots, large_wait_ms)
        _check(lib.mh_server_create(ctypes.byref(o), ctypes.byref(self.ptr)))

    def submit(self, bitmaps, G, Nt, Nn, h, alpha=(1, 10)) -> int:
        bm = np.ascontiguousarray(bitmaps, dtype=np.uint64)
        t = ctypes.c_uint64()
        _check(load().mh_submit(self.ptr, bm.ctypes.data, G, Nt, Nn, h, mh_rational(*alpha), ctypes.byref(t)))
        return t.value

    def cancel(self, ticket) -> None:
        _check(load().mh_cancel(self.ptr, ticket))

    def poll(self, ticket):
        """Result if finished, None while queued or running."""
        p = ctypes.POINTER(mh_result)()
        rc = load().mh_poll(self.ptr, ticket, ctypes.byref(p))
        if rc == MH_EAGAIN:
            return None
        _check(rc)
        return _to_result(p)

    def wait(self, ticket, timeout_ms: int = -1):
        p = ctypes.POINTER(mh_result)()
        rc = load().mh_wait(self.ptr, ticket, timeout_ms, ctypes.byref(p))
        if rc == MH_EAGAIN:
            return None
        _check(rc)
        return _to_result(p)

    def stats(self):
        a, q, b, m = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(load().mh_server_stats(self.ptr, ctypes.byref(a), ctypes.byref(q), ctypes.byref(b), ctypes.byref(m)))
        return {"launches": a.value, "queued": q.value, "active": b.value, "bytes_in_use": m.value}

    def close(self):
        if self.ptr:
            load().mh_server_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
