"""The multi-process path of the benchmark on the host (gloo, world size 2):
barrier, the maximum of the per-rank times, the whole-job throughput (replicas:
units of all ranks over the slowest rank's time), and the reference arm's rule
that only rank 0 runs and prints."""
import io
import os
import sys
from contextlib import redirect_stdout

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r = bench.Ranks(world, rank, "cpu", dist)
        r.barrier()
        ms_local = 10.0 * (rank + 1)  # rank 1 is the slow one
        value, ms = r.throughput(units_per_rank=8 * 5, ms_local=ms_local)
        r.barrier()
        out[rank] = (value, ms)
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_units():
    world, port = 2, 29500 + os.getpid() % 1000
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        value, ms = out[rank]
        assert ms == 20.0
        assert abs(value - world * 40 / 0.020) < 1e-9  # 80 view iterations in 20 ms


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(1, 0, "cpu")
    r.barrier()
    assert r.max(3.5) == 3.5
    assert r.throughput(10, 5.0) == (2000.0, 5.0)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup = 1, 0

    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(Args(), rank=1, world=2) == 0
    assert buf.getvalue() == ""
