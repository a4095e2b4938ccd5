"""The N>1 path on CPU: two gloo ranks, each with its own independent unit of
work; the job time is the max over ranks and the throughput counts the units
of all ranks (bench.max_over_ranks / job_throughput).  No GPU."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 30.0][rank]                 # the second rank is slower
    got = bench.max_over_ranks(ms)
    q.put((rank, got, bench.job_throughput(1_000_000, world, got)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max():
    import random
    port = 29500 + random.randint(0, 2000)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [30.0, 30.0]
    # 2 ranks x 1e6 units in 30 ms = 66.67 Mops/s
    assert all(abs(r[2] - 2e6 / 0.03 / 1e6) < 1e-6 for r in res)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0) == 7.0
    assert bench.job_throughput(10, 1, 1.0) == pytest.approx(0.01)
