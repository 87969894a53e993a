"""Multi-rank logic of the benchmark on CPU (gloo, world size 2): the timing
aggregate is the max over ranks and batch sharding is a disjoint cover."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = bench.max_over_ranks(10.0 + rank)
        mine = bench.shard(11, rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out[rank] = (m, gathered)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_sharding_gloo_world2():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        m, gathered = res[r]
        assert m == 11.0
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(11))
        assert not set(gathered[0]) & set(gathered[1])


def test_single_process_identity():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
