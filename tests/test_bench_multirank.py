"""The N > 1 path of bench.py on CPU: replicas on two gloo ranks.  Whole-job
throughput = units summed over ranks / the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = [100.0, 300.0][rank]
    secs = [2.0, 5.0][rank]
    value, tmax, total = bench.aggregate_over_ranks(units, secs)
    out[rank] = (value, tmax, total)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        value, tmax, total = out[r]
        assert tmax == 5.0 and total == 400.0
        assert value == pytest.approx(80.0)


def test_single_process_aggregate():
    import bench
    assert bench.aggregate_over_ranks(10.0, 2.0) == (5.0, 2.0, 10.0)
