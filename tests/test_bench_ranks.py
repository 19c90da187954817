"""bench.py's multi-rank plumbing on CPU: two gloo ranks agree on the max-over-ranks
time (the value every rank's whole-job throughput is computed from), pass the
barrier, and a non-zero rank of the CPU reference arm exits without work."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [10.0 * (rank + 1), 5.0 - rank]
        bench.barrier(world)
        got = bench.aggregate_max(local, world)
        steps = 4
        value = world * steps / (got[0] / 1e3)
        q.put((rank, got, value, bench._dist_env()))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value, env in out:
        assert got == [20.0, 5.0]          # max over ranks of each entry
        assert value == pytest.approx(2 * 4 / 0.020)   # all ranks' solves / the slowest rank's time
        assert env == (rank, 2, rank)


def test_single_rank_aggregate_is_identity():
    assert bench.aggregate_max([1.5, 2.5], 1) == [1.5, 2.5]
    bench.barrier(1)


def test_reference_arm_nonzero_rank_does_no_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.main(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]) == 0
    assert capsys.readouterr().out == ""
