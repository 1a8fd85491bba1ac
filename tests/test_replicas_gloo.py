"""The N > 1 host logic (sharding of independent problems, max/sum over
ranks) with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2607_23354_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = replicas.rank_world()
    mine = replicas.shard(range(4096), r, w)
    total = replicas.sum_over_ranks(len(mine))
    worst = replicas.max_over_ranks(1.5 + r)
    dist.barrier()
    out[rank] = (r, w, lr, mine[:3], len(mine), total, worst)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][:3] == (0, 2, 0) and res[1][:3] == (1, 2, 1)
    assert res[0][3] == [0, 2, 4] and res[1][3] == [1, 3, 5]
    assert res[0][4] + res[1][4] == 4096
    assert res[0][5] == res[1][5] == 4096.0
    assert res[0][6] == res[1][6] == 2.5


def test_single_process_is_identity():
    assert replicas.shard([1, 2, 3], 0, 1) == [1, 2, 3]
    assert replicas.max_over_ranks(3.0) == 3.0
