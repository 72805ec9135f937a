"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, no data-path
collective), each timing its own run; the job's time is the slowest rank's
and the whole-job rate counts every rank's units."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 10.0 + 5.0 * rank                 # rank 1 is the slow one
    ms = bench.max_over_ranks(ms_local, dist, "cpu")
    rate = bench.whole_job_rate(100.0, ms, world)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ms, rate))


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_units():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in res:
        assert ms == 15.0
        assert rate == pytest.approx(100.0 * 2 / 0.015)


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.whole_job_rate(10.0, 2.0, 1) == pytest.approx(5000.0)
