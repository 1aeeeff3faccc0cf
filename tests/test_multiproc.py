"""The N>1 benchmark path on CPU: two gloo ranks shard value sets and reduce timings."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = bench.rank_seeds(rank, 64)
    mine = [10.0 + rank, 5.0 * (1 + rank), 1.0, 2.0 - rank]
    red = bench.max_over_ranks(mine, dist, "cpu")
    out[rank] = (seeds[0], seeds[-1], red)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert out[0][:2] == (0, 63) and out[1][:2] == (64, 127)     # disjoint contiguous seed ranges
    for r in range(world):
        assert out[r][2] == [11.0, 10.0, 1.0, 2.0]                # element-wise max over ranks


def test_parallel_oracle_baseline_small():
    # the bench's CPU baseline: one oracle process per core, all started together
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    walls = bench.oracle_parallel(3000, 2, rounds=2)
    assert len(walls) == 2 and all(w > 0.0 for w in walls)
