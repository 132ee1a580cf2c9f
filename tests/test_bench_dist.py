"""The benchmark's multi-rank path (barrier, max over ranks, whole-job value)
on two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, _ = bench.dist_init("gloo")
    assert (r, w) == (rank, world)
    bench.barrier(w)
    t = bench.max_over_ranks(1.0 + rank, w)          # rank 1 is the slower one
    out[rank] = (t, bench.aggregate_mlups(1000, 10, t, w))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_and_aggregate():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        t, v = out[rank]
        assert t == 2.0
        assert v == pytest.approx(world * 1000 * 10 / 2.0 / 1e6)
