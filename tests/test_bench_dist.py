"""The bench's multi-rank aggregation (max time over ranks, summed work) on 2 gloo ranks (CPU)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank)          # rank 1 is the slow one
    s = bench.sum_over_ranks(10.0 * (rank + 1))   # work adds up
    bench.barrier()
    out[rank] = (t, s, bench.rank_info())
    dist.destroy_process_group()


def test_two_rank_aggregation():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        t, s, info = out[r]
        assert t == 2.0 and s == 30.0 and info == (r, r, 2)
