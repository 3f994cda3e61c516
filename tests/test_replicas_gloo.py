"""The N > 1 benchmark path (independent replicas, one event per rank): the
max-over-ranks time and the summed units, run as world-size-2 gloo ranks on
the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r timed 100 + 50 r ms for (1000 + r) clusters x 10 steps
    ms, units, rate = bench.aggregate(100.0 + 50.0 * rank, (1000 + rank) * 10, dist, "cpu")
    dist.barrier()
    q.put((rank, ms, units, rate))
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, rate in out:
        assert ms == 150.0                       # the slowest rank
        assert units == 20010.0                  # every rank's clusters
        assert abs(rate - 20010.0 / 0.150) < 1e-6


def test_aggregate_single_process_is_identity():
    import bench
    assert bench.aggregate(200.0, 5000) == (200.0, 5000, 25000.0)
