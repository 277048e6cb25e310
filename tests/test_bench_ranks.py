"""bench.py's multi-rank host logic with two gloo ranks on the CPU: the
timed total is the slowest rank's, and the whole-job time per map divides it
by the maps all ranks ran (independent replicas, no data-path collective)."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 100.0 + 50.0 * rank  # rank 1 is slower
        total = bench.max_over_ranks(mine, torch.device("cpu"))
        per_step, per_map = bench.replica_throughput(total, steps=10, world=world)
        out.put((rank, total, per_step, per_map))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_total():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, per_step, per_map in res:
        assert total == 150.0
        assert per_step == 15.0
        assert per_map == 7.5


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.replica_throughput(30.0, 10, 1) == (3.0, 3.0)
