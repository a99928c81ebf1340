"""The multi-GPU bench path runs independent replicas (one grid per rank, no data-path
exchange): whole-job value = sum of cell-updates / slowest rank's time.  Checked with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 150.0][rank]
    units = [1.0e9, 1.2e9][rank]
    q.put((rank, bench.aggregate(ms, units, dist, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        ms, units = res[r]
        assert ms == pytest.approx(150.0)
        assert units == pytest.approx(2.2e9)


def test_single_process_aggregation():
    import bench

    assert bench.aggregate(10.0, 5.0) == (10.0, 5.0)
