"""The bench's multi-rank path (replicas, weak scaling) on CPU: two gloo ranks
on 127.0.0.1. The slowest rank's time sets the job time and the throughput
counts every rank's work."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.rank_env()
    ms = bench.max_over_ranks(100.0 + 50.0 * r, w)  # rank 1 is slower
    rate = bench.aggregate_rate(1_000_000, 4, w, ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, lr, ms, rate))


def test_two_gloo_ranks_take_max_time_and_sum_work():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, ms, rate) in enumerate(out):
        assert (rank, world, local) == (r, 2, r)
        assert ms == 150.0
        assert rate == pytest.approx(1_000_000 * 4 * 2 / 0.150 / 1e9)


def test_single_rank_defaults(monkeypatch):
    import bench

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.rank_env() == (0, 1, 0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
