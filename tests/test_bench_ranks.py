"""The N > 1 path of bench.py on CPU: two gloo ranks, each a replica with its own time; the
reported time is the slowest rank's and the value counts the steps of every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank                   # rank 1 is the slowest
    slowest = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (slowest, bench.whole_job_rate(world, 10, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time_and_the_whole_job_rate():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        slowest, rate = out[r]
        assert slowest == 150.0
        assert abs(rate - 2 * 10 / 0.150) < 1e-9
