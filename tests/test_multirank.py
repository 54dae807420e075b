"""The benchmark's host-side contract on CPU: multi-rank logic with the gloo
backend (world size 2: each rank runs an independent replica; the whole-job
rate is the work of all ranks over the slowest rank's time), and the
reference arm's JSON line."""
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


@pytest.mark.slow
def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores, on the
    benchmark workload itself) prints one JSON line with the keys of the
    benchmark contract, its own cpu_baseline and an e2e entry without copies;
    under a launcher, ranks other than 0 print nothing and exit 0."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "256x128x128" in d["config"]["workload"]
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r1 = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=root, env=env)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
