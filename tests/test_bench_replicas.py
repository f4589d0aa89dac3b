"""bench.py runs N independent replicas (one per GPU, no data-path collective); its
timing plumbing -- a barrier around the timed region and the maximum of the per-rank
times -- is checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as tmp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    dist = bench.dist_init(ws, "gloo")
    bench.barrier(ws)
    t = bench.reduce_max(1.5 + rank, ws)
    out[rank] = t
    dist.destroy_process_group()


def test_two_rank_max_and_barrier():
    world = 2
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == 2.5


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.25, 1) == 3.25
    bench.barrier(1)
