"""The N > 1 path of bench.py is independent replicas: the job's time is the
slowest rank's and the job's throughput counts every rank.  Checked with two
gloo ranks on CPU (no GPU, no data-path collective)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def reduce_max(v):
        t = torch.tensor([v], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    local_ms = 10.0 * (rank + 1)          # rank 1 is the slow one
    value, ms = bench.whole_job_throughput(local_ms, dof_per_rank=1000, steps=4, world=world, reduce_max=reduce_max)
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_slowest_rank_and_total_work():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()   # no fork of a process that may hold threads
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1]
    value, ms = out[0]
    assert ms == 20.0
    assert value == pytest.approx(world * 1000 * 4 / 0.020)
