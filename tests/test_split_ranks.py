"""The split solve's round protocol (paper_2603_16721_gb300/split.py) on CPU ranks:
two and three gloo processes each search their shard of every round's depth-1
genes with the threaded CPU P-DFS (a stand-in for the GPU shard, itself checked
against the oracle), exchange their round results with the library's gather and
merge, and commit the merged round.  The selections and the per-round counters
must be those of the unsplit oracle P-DFS."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_2603_16721_gb300 import split
from test_oracle_pins import _random_cohort


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleShard:
    """search / commit of one rank's shard, on the CPU."""

    def __init__(self, bm, G, Nt, Nn, h, alpha, rank, world):
        self.a = (bm, G, Nt, Nn)
        self.h, self.alpha, self.rank, self.world = h, alpha, rank, world
        self.order = oracle.sparsity_order(bm, G, Nt, Nn)
        self.U = oracle.full_tumor_mask(Nt)
        self.done = Nt == 0
        self.records, self.visited, self.pruned = [], [], []

    def search(self):
        z = np.zeros(self.h, dtype=np.uint64)
        if self.done:
            return {"done": True, "have": False, "score": 0, "genes": (0,) * self.h, "visited": z, "pruned": z}
        r = oracle.mt_round(*self.a, self.h, self.U, self.alpha, order=self.order, threads=1, shard=self.rank,
                            nshards=self.world)
        return {"done": False, "have": r.have, "score": r.score, "genes": r.genes if r.have else (0,) * self.h,
                "visited": r.visited, "pruned": r.pruned}

    def commit(self, m):
        self.visited.append(np.asarray(m["visited"], dtype=np.uint64))
        self.pruned.append(np.asarray(m["pruned"], dtype=np.uint64))
        if not m["have"]:
            self.done = True
            return True
        genes = np.array([m["genes"]], dtype=np.int32)
        tp, fp = oracle.cover_counts(*self.a, genes, self.U)
        self.records.append((tuple(m["genes"]), int(tp[0]), int(fp[0])))
        self.U = oracle.delcols(*self.a, m["genes"], self.U)
        self.done = not self.U.any()
        return self.done


def _rank_main(rank, world, port, cases, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = []
        for bm, G, Nt, Nn, h, alpha in cases:
            sh = OracleShard(bm, G, Nt, Nn, h, alpha, rank, world)
            rounds = split.run_rounds(sh.search, sh.commit, split.torch_gather(), h)
            out.append((sh.records, np.array(sh.visited).reshape(-1, h), np.array(sh.pruned).reshape(-1, h), rounds))
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def _cases():
    rng = np.random.default_rng(4242)
    cases = []
    for i in range(6):
        h = int(rng.integers(1, 5))
        G = int(rng.integers(max(h, 2), 40 if h <= 3 else 24))
        Nt, Nn = int(rng.integers(1, 150)), int(rng.integers(0, 80))
        bm, _, _ = _random_cohort(rng, G, Nt, Nn, rng.uniform(0.05, 0.4), rng.uniform(0.0, 0.3))
        cases.append((bm, G, Nt, Nn, h, [(1, 10), (3, 7), (1, 1)][i % 3]))
    c = synth.generate(synth.c2_law(400, 120, 60, seed=9, h=3))
    cases.append((c.bitmaps, c.G, c.Nt, c.Nn, 3, (1, 10)))
    cases.append((np.zeros((2, 2), dtype=np.uint64), 2, 10, 10, 3, (1, 10)))  # G < h
    return cases


@pytest.mark.parametrize("world", [2, 3])
def test_split_rounds_equal_unsplit_oracle(world):
    cases = _cases()
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, cases, q)) for r in range(world)]
    for p in procs:
        p.start()
    outs = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for i, (bm, G, Nt, Nn, h, alpha) in enumerate(cases):
        ref = oracle.pdfs(bm, G, Nt, Nn, h, alpha)
        for rank in range(world):  # every rank holds the same merged result
            recs, vis, pru, rounds = outs[rank][i]
            assert recs == ref.records()
            assert rounds == ref.visited.shape[0]
            assert np.array_equal(vis, ref.visited) and np.array_equal(pru, ref.pruned)


def test_merge_picks_largest_score_then_smallest_tuple():
    z = np.zeros(3, dtype=np.uint64)
    parts = [{"done": False, "have": True, "score": 50, "genes": (4, 7, 9), "visited": z + 1, "pruned": z},
             {"done": False, "have": True, "score": 50, "genes": (4, 6, 11), "visited": z + 2, "pruned": z + 1},
             {"done": False, "have": False, "score": 0, "genes": (0, 0, 0), "visited": z + 3, "pruned": z + 3},
             {"done": False, "have": True, "score": 49, "genes": (0, 1, 2), "visited": z, "pruned": z}]
    m = split.merge(parts, 3)
    assert m["have"] and m["score"] == 50 and m["genes"] == (4, 6, 11)
    assert m["visited"].tolist() == [6, 6, 6] and m["pruned"].tolist() == [4, 4, 4]
    big = np.array([2 ** 64 - 1] * 3, dtype=np.uint64)
    w = split.merge([dict(parts[0], visited=big), dict(parts[1], visited=z + 2)], 3)
    assert w["visited"].tolist() == [1, 1, 1]  # modulo 2^64, like the counters
    v = split.pack(parts[1], 3)
    assert split.unpack(v, 3)["genes"] == (4, 6, 11)
