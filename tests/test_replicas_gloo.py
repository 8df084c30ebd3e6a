"""The N > 1 path of bench.py is replicas only: each rank solves its own copy
and the job reports (sum of units) / (max time over ranks).  Checked with two
gloo ranks on the CPU."""
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


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = 1000.0 * (rank + 1)          # rank r processed 1000 (r+1) units
    seconds = 2.0 + rank                  # and took 2 + r seconds
    value, sec = bench.replica_aggregate(units, seconds, world, "cpu")
    out[rank] = (value, sec)
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        value, sec = out[r]
        assert sec == pytest.approx(3.0)                  # max over ranks
        assert value == pytest.approx(3000.0 / 3.0)       # all units / max time


def test_single_process_aggregation_is_plain_ratio():
    import bench
    assert bench.replica_aggregate(10.0, 4.0, 1) == (2.5, 4.0)
