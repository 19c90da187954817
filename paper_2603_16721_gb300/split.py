"""One greedy solve split over the ranks of a process group (the lambda split of
§III-E): every rank searches its share of each round's depth-1 genes on its own
GPU (``mh_shard_search``), the ranks all-gather their best candidates and counter
shares, every rank merges them the same way (largest score, ties to the smallest
ascending tuple of original indices; counters summed modulo 2^64) and applies
the merged winner (``mh_shard_commit``).  The exchange per round is a few hundred
bytes; no data-path memory moves between GPUs.

``run_rounds`` is the round loop over any ``search`` / ``commit`` / ``gather``
triple (the library's shards on a GPU; other searchers in tests); ``split_solve``
wires it to the library and ``torch.distributed``.
"""
from __future__ import annotations

import numpy as np

from . import mh

_MAXH = 9
_LEN = 3 + 3 * _MAXH  # done, have, score, genes, visited, pruned


def pack(rb: dict, h: int) -> np.ndarray:
    """A round result as one int64 vector (counters as their 64-bit patterns)."""
    v = np.zeros(_LEN, dtype=np.int64)
    v[0], v[1], v[2] = int(rb["done"]), int(rb["have"]), int(rb["score"])
    v[3:3 + h] = np.asarray(rb["genes"][:h], dtype=np.int64)
    v[3 + _MAXH:3 + _MAXH + h] = np.asarray(rb["visited"][:h], dtype=np.uint64).view(np.int64)
    v[3 + 2 * _MAXH:3 + 2 * _MAXH + h] = np.asarray(rb["pruned"][:h], dtype=np.uint64).view(np.int64)
    return v


def unpack(v: np.ndarray, h: int) -> dict:
    v = np.asarray(v, dtype=np.int64)
    return {"done": bool(v[0]), "have": bool(v[1]), "score": int(v[2]),
            "genes": tuple(int(g) for g in v[3:3 + h]),
            "visited": v[3 + _MAXH:3 + _MAXH + h].view(np.uint64).copy(),
            "pruned": v[3 + 2 * _MAXH:3 + 2 * _MAXH + h].view(np.uint64).copy()}


def merge(parts: list, h: int) -> dict:
    """The round over all ranks: the best candidate (score desc, then the smallest
    ascending tuple of original indices, §III-D's strict comparison in original
    order) and the counters summed (u64, wrapping like the counters themselves)."""
    best = None
    for p in parts:
        if p["have"] and (best is None or (p["score"], tuple(-g for g in p["genes"])) >
                          (best["score"], tuple(-g for g in best["genes"]))):
            best = p
    visited = np.zeros(h, dtype=np.uint64)
    pruned = np.zeros(h, dtype=np.uint64)
    with np.errstate(over="ignore"):
        for p in parts:
            visited += np.asarray(p["visited"], dtype=np.uint64)
            pruned += np.asarray(p["pruned"], dtype=np.uint64)
    return {"done": all(p["done"] for p in parts), "have": best is not None,
            "score": best["score"] if best else 0, "genes": best["genes"] if best else tuple([0] * h),
            "visited": visited, "pruned": pruned}


def run_rounds(search, commit, gather, h: int) -> int:
    """Round loop: search the local share, gather every rank's share, merge, commit
    the merged round on every rank.  Returns the number of rounds searched."""
    rounds = 0
    while True:
        parts = gather(search())
        merged = merge(parts, h)
        if merged["done"]:
            return rounds
        rounds += 1
        if commit(merged):
            return rounds


def torch_gather(group=None, device="cpu"):
    """An all-gather of round results over a torch.distributed group."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)

    def gather(rb):
        h = len(rb["genes"])
        t = torch.from_numpy(pack(rb, h)).to(device)
        out = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(out, t, group=group)
        return [unpack(o.cpu().numpy(), h) for o in out]

    return gather


def split_solve(handle: "mh.Handle", h: int, alpha=(1, 10), prune: int = mh.MH_PRUNE_PAPER, group=None,
                device="cpu") -> "mh.Result":
    """The solve of ``handle`` split over the ranks of ``group`` (this rank's shard =
    its rank); every rank returns the same result."""
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    with mh.Shard(handle, h, alpha, rank, world, prune) as X:
        run_rounds(X.search, X.commit, torch_gather(group, device), h)
        return X.result()
