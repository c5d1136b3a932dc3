"""The multi-rank host logic of bench.py on CPU with gloo, world size 2: the
max-over-ranks timing reduction and the round-robin sharding of independent
problems (every problem exactly once, no exchange)."""
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
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks(1.5 + rank, world)
        mine = bench.shard(64, rank, world)
        got = [None] * world
        dist.all_gather_object(got, mine)
        if rank == 0:
            flat = sorted(i for part in got for i in part)
            out[world] = float(flat == list(range(64)) and all(len(p) == 32 for p in got))
    finally:
        dist.destroy_process_group()


def test_bench_rank_logic_gloo_world2():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == 2.5
    assert out[world] == 1.0


def test_bench_rank_logic_single_process():
    import bench

    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert bench.shard(5, 1, 2) == [1, 3]
