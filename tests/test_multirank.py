"""The benchmark's replica path on a world of two gloo ranks on the CPU: the
max step time over ranks, the replica throughput, and each rank's own
workload (its seeded trajectory of the shared model) stepped end to end, with
the FP64 oracle standing in for the rank's GPU."""
import os

import numpy as np
import pytest
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
    q.put(("agg", rank, ms, value))
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
    for _, rank, ms, value in res:
        assert ms == pytest.approx(2.0)
        assert value == pytest.approx(2 * 1e3 / 2.0)


N, STEPS = 24, 12


def _replica_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import time

    import bench
    import oracle
    import synth

    oracle.set_threads(1)
    seed = synth.seed_for(2)
    C, factors, a = bench.workload(N, N, seed, "cpu")
    u0 = bench.replica_initial_state(N, seed, rank)
    rom = oracle.Rom("full", N, a, bench.NU, bench.DT, C=C.numpy())
    h = rom.initial_history(u0[0])
    dist.barrier()
    t0 = time.perf_counter()
    rom.step(h, STEPS)
    ms = (time.perf_counter() - t0) * 1e3 / STEPS
    dist.barrier()
    ms_max = bench.max_over_ranks(ms, device="cpu")
    q.put(("replica", rank, u0[0], h[:N].copy(), ms, ms_max, bench.replica_throughput(ms_max, world)))
    dist.destroy_process_group()


def test_two_rank_replicas_step_their_own_trajectories():
    import bench
    import oracle
    import synth

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_replica_worker, args=(r, 2, 29519, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in range(2)], key=lambda x: x[1])
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    seed = synth.seed_for(2)
    C, _, a = bench.workload(N, N, seed, "cpu")
    # the ranks stepped different trajectories of the same model
    assert not np.array_equal(res[0][2], res[1][2])
    for _, rank, u0, final, ms, ms_max, value in res:
        np.testing.assert_array_equal(u0, synth.initial_condition(N, seed, traj=rank)[0])
        ref = oracle.Rom("full", N, a, bench.NU, bench.DT, C=C.numpy())
        h = ref.initial_history(u0)
        ref.step(h, STEPS)
        np.testing.assert_array_equal(final, h[:N])
        # every rank reports the slowest rank's time and the throughput of both replicas
        assert ms_max == pytest.approx(max(r[4] for r in res))
        assert value == pytest.approx(2 * 1e3 / ms_max)
