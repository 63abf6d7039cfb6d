"""The N > 1 path of bench.py on CPU: two gloo ranks, max-over-ranks timing and the whole-job
rate of weak scaling (every rank runs its own copy of the workload)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [2.0, 3.5][rank]  # this rank's time for its steps
    slowest = bench.max_over_ranks(dist, local)
    dist.barrier()
    rate = bench.whole_job_rate(1000.0, 4, world, slowest)
    out.put((rank, slowest, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_rate():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in res:
        assert slowest == 3.5
        assert rate == 2 * 1000.0 * 4 / 3.5
