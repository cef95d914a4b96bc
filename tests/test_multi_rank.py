"""The benchmark's multi-GPU form is replicas only (no collective on the data path): each rank
runs the whole workload and the job's rate is every rank's units over the slowest rank's time.
This runs that aggregation as two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r "took" 2 + r seconds for 100 units
    rate, slowest = bench.job_throughput(2.0 + rank, 100.0)
    out[rank] = (rate, slowest)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_rate_is_total_units_over_slowest_rank():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        rate, slowest = res[rank]
        assert slowest == pytest.approx(3.0)
        assert rate == pytest.approx(world * 100.0 / 3.0)


def test_single_process_rate():
    import bench
    rate, t = bench.job_throughput(4.0, 100.0)
    assert t == 4.0 and rate == pytest.approx(25.0)
