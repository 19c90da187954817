"""The split solve through the C ABI: two gloo ranks (processes) on the GPU, each
searching its shard of every round's depth-1 genes (mh_shard_search), exchanging
round results between kernel launches on the host, and committing the merged
round (mh_shard_commit).  No kernel waits on another rank: every exchange happens
between launches.  Both ranks must end with the selections and the per-round
counters of the unsplit solve and of the oracle."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cohorts():
    return [(synth.generate(synth.c2_law(1500, 300, 200, seed=41, h=3)), 3),
            (synth.generate(synth.c3_law(1200, 400, 200, seed=42, h=4)), 4),
            (synth.generate(synth.c1()), 2)]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        from paper_2603_16721_gb300 import mh, split
        out = []
        for c, h in _cohorts():
            with mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) as H:
                r = split.split_solve(H, h, (1, 10))
            out.append((r.records(), r.visited, r.pruned))
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_ranks_equal_unsplit_solve():
    import torch.multiprocessing as mp
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_16721_gb300 import mh
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    outs = dict(q.get(timeout=600) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for i, (c, h) in enumerate(_cohorts()):
        with mh.mh_create(c.bitmaps, c.G, c.Nt, c.Nn) as H:
            ref = mh.mh_solve_ex(H, h, (1, 10), mode=mh.MH_MODE_LAUNCHES)
        orc = oracle.pdfs_mt(c.bitmaps, c.G, c.Nt, c.Nn, h, (1, 10))
        assert ref.records() == orc.records()
        for rank in range(world):
            recs, vis, pru = outs[rank][i]
            assert recs == ref.records()
            assert np.array_equal(vis, ref.visited) and np.array_equal(pru, ref.pruned)
            assert np.array_equal(vis, orc.visited) and np.array_equal(pru, orc.pruned)
