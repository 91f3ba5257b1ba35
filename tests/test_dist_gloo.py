"""The multi-replica host logic of bench.py on CPU with two gloo ranks: the
timed region is the slowest rank's, and the job value counts every replica's
node updates (independent replicas, no data-path collective)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 180.0][rank]                  # rank 1 is the slower replica
    m = bench.max_over_ranks(ms)
    v = bench.job_glups(world, 1_000_000, 100, m)
    r, w, lr = bench.dist_env()
    out.put((rank, m, v, r, w, lr))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v, r, w, lr in res:
        assert m == 180.0 and r == rank and w == 2 and lr == rank
        assert v == pytest.approx(2 * 1e6 * 100 / 0.18 / 1e9)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_glups(1, 10, 10, 1.0) == pytest.approx(1e-4)
