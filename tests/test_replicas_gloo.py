"""Multi-rank path of the benchmark on CPU: independent replicas, one per
rank, combined as total work / slowest rank (gloo, world size 2)."""
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


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r pretends to need (r + 1) seconds for 100 units
    value, t = bench.aggregate_throughput(float(rank + 1), 100.0, world, "cpu")
    out[rank] = (value, t)
    dist.destroy_process_group()


def test_replica_throughput_is_total_work_over_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, t = res[rank]
        assert t == pytest.approx(2.0)
        assert value == pytest.approx(200.0 / 2.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.aggregate_throughput(2.0, 50.0, 1) == (25.0, 2.0)
