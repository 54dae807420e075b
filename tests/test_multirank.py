"""Multi-rank bench logic on CPU with the gloo backend (world size 2): each
rank runs an independent replica; the whole-job rate is the work of all
ranks over the slowest rank's time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ms_local = 100.0 * (rank + 1)  # rank 1 is the slow one
    rate, ms_max = bench.job_rate(1_000_000, 10, ms_local, world, reduce_max)
    out[rank] = (rate, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_uses_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    for r in range(world):
        rate, ms_max = out[r]
        assert ms_max == pytest.approx(200.0)
        assert rate == pytest.approx(1_000_000 * 2 * 10 / 0.2 / 1e6)
