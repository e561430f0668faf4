"""World-size-2 gloo test of the instance sharding used by bench.py (CPU only): disjoint
identity ranges, the max-over-ranks job time and the summed unit count."""
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
    import torch
    import torch.distributed as dist

    from paper_2512_16543_gb300 import sharding
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ids = sharding.shard_ids(rank, world, 4)
    t = sharding.max_over_ranks(1.5 + rank)           # rank 1 is the slow one
    n = sharding.sum_over_ranks(len(ids))
    gathered = [None] * world
    dist.all_gather_object(gathered, ids)
    out[rank] = (ids, t, n, gathered)
    dist.destroy_process_group()


def test_two_rank_sharding():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    ids0, t0, n0, g0 = out[0]
    ids1, t1, n1, _ = out[1]
    assert ids0 == [0, 1, 2, 3] and ids1 == [4, 5, 6, 7]
    assert set(g0[0]).isdisjoint(g0[1])
    assert t0 == t1 == 2.5
    assert n0 == n1 == 8


def test_single_process_passthrough():
    from paper_2512_16543_gb300 import sharding
    assert sharding.max_over_ranks(3.0) == 3.0
    assert sharding.shard_ids(0, 1, 3) == [0, 1, 2]
    with pytest.raises(ValueError):
        sharding.shard_ids(2, 2, 3)
