"""bench.py's multi-GPU form runs independent replicas; its only exchange is
the whole-job aggregation (max time over ranks, summed tokens).  Checked
with two gloo ranks on the CPU."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, tokens = bench.reduce_over_ranks(10.0 * (rank + 1), 1000.0 * (rank + 1), "cpu")
    out[rank] = (ms, tokens)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_reduce_over_ranks(world):
    port = 29500 + world * 7 + os.getpid() % 500
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    expect = (10.0 * world, 1000.0 * world * (world + 1) / 2)
    assert all(out[r] == expect for r in range(world))
