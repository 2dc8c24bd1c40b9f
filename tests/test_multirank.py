"""The benchmark's multi-rank aggregation (max step time over ranks, replica
throughput) on a world of two gloo ranks on the CPU."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms_local = 1.0 + rank  # rank 1 is slower
    ms = bench.max_over_ranks(ms_local, device="cpu")
    value = bench.replica_throughput(ms, world)
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29517
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == pytest.approx(2.0)
        assert value == pytest.approx(2 * 1e3 / 2.0)
