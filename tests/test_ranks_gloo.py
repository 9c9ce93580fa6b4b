"""The benchmark's multi-rank path on CPU: two gloo ranks, barrier, max-over-ranks time and
whole-job (summed) throughput, as bench.py uses them under torchrun (weak scaling, no data-path
collective)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    ranks = bench.Ranks(backend="gloo")
    assert ranks.on and ranks.world == world and ranks.rank == rank
    ranks.barrier()
    # rank r evaluated 100 * (r + 1) particles in 1 + r seconds
    value, slowest = bench.aggregate(ranks, 100.0 * (rank + 1), 1.0 + rank)
    out[rank] = (value, slowest)
    ranks.dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_weak_scaling():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        value, slowest = out[r]
        assert slowest == pytest.approx(2.0)              # max over ranks
        assert value == pytest.approx(300.0 / 2.0)        # all ranks' units / slowest rank's time


def test_single_rank_needs_no_process_group(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    r = bench.Ranks()
    assert not r.on
    assert bench.aggregate(r, 50.0, 2.0) == (25.0, 2.0)
