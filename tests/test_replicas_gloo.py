"""The multi-GPU path of the benchmark is replicas only: every rank decodes
the same workload on its own GPU with no collective on the data path, and
the job's time is the slowest rank's.  The rank aggregation runs here on
CPU with two gloo ranks."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, torch.device("cpu"))
    out[rank] = (ms, bench.job_throughput(1000.0, world, ms / 1000.0))
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_max_over_ranks_and_rate_sums_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    # both ranks see the slower rank's 15 ms; 2 ranks x 1000 units / 15 ms
    for r in range(2):
        ms, rate = out[r]
        assert ms == 15.0
        assert abs(rate - 2000.0 / 0.015) < 1e-6 * rate


def test_single_process_needs_no_process_group():
    torch = pytest.importorskip("torch")
    import bench
    assert bench.max_over_ranks(7.5, torch.device("cpu")) == 7.5
    assert bench.job_throughput(10.0, 1, 2.0) == 5.0
