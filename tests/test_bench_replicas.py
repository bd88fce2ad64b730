"""The N > 1 path of bench.py runs independent replicas: the whole-job time is the slowest rank's,
the work is the sum over ranks. Checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, b = bench.aggregate(10.0 + 5.0 * rank, 100.0 * (rank + 1), dist, "cpu")
    out[rank] = (t, b)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == (15.0, 300.0) and out[1] == (15.0, 300.0)


def test_single_rank_passthrough():
    import bench
    assert bench.aggregate(3.5, 42.0, None, "cpu") == (3.5, 42.0)
