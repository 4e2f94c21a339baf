"""The benchmark's multi-rank path on CPU: two gloo ranks, each timing its own
replica of the workload; the job's step time is the max over ranks and the
throughput counts every rank's units (weak scaling, no data-path collective)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    import bench
    total = bench.max_over_ranks(100.0 + 25.0 * rank, dist, torch.device("cpu"))
    rate = bench.job_rate(units_per_rank=1000, world=world, steps=4, total_ms=total)
    out.put((rank, total, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_step_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in results] == [125.0, 125.0]
    # 2 ranks x 1000 units x 4 steps in 125 ms
    assert all(abs(r[2] - 64000.0) < 1e-6 for r in results)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(7.5, None, None) == 7.5
    assert bench.job_rate(10, 1, 2, 1000.0) == 20.0
