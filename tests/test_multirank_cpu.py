"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own replica; the job
reports the slowest rank's time and the work of all ranks (weak scaling, replicas only)."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [10.0, 25.0][rank]
    pushes = [1000.0, 3000.0][rank]
    res = bench.aggregate(ms, pushes, 4, world)
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    world, port = 2, 29500 + os.getpid() % 1000
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms_max, total, value = res[r]
        assert ms_max == 25.0
        assert total == (1000.0 + 3000.0) * 4
        assert value == pytest.approx(total / 0.025)


def test_single_rank_aggregation():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(5.0, 200.0, 10, 1) == (5.0, 2000.0, 2000.0 / 0.005)
