"""The N > 1 path of bench.py (replicas, no data-path collective): two gloo ranks on the CPU check
that the whole-job value is the work of all ranks over the slowest rank's timed region."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 + 50.0 * rank            # rank 1 is the slowest
    work_local = 1.0e9 * (rank + 1)
    value, ms_max = bench.aggregate(torch, dist, ms_local, work_local, world, "cpu")
    out[rank] = (value, ms_max)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        value, ms_max = res[r]
        assert ms_max == 150.0
        assert value == pytest.approx((1.0e9 + 2.0e9) / 0.150)
