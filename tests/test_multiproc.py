"""The N-GPU bench path runs independent replicas (one per rank) and reports
the units of all ranks over the slowest rank's time.  Its rank aggregation is
exercised here with two gloo ranks on the CPU."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = [0.5, 0.75][rank]
    units = [100, 300][rank]
    t, u = bench.aggregate_over_ranks(elapsed, units, world)
    q.put((rank, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_total_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 0.75, 400.0), (1, 0.75, 400.0)]


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_over_ranks(1.5, 42, 1) == (1.5, 42)
