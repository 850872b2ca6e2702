"""Multi-process host logic on CPU: two gloo ranks (no GPU)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2310_14712_gb300 import replicas


def test_shard_columns_covers_every_column_once():
    for ncols in (0, 1, 5, 64, 65):
        for world in (1, 2, 3, 8):
            cols = [c for r in range(world) for c in replicas.shard_columns(ncols, r, world)]
            assert cols == list(range(ncols))
            sizes = [len(replicas.shard_columns(ncols, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard_columns(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, rk, _ = replicas.dist_env()
        assert (ws, rk) == (world, rank)
        replicas.barrier(ws)
        # Per-rank "time" and the job-wide maximum; per-rank work and its sum.
        t = replicas.reduce_max(1.5 + rank, ws)
        mine = list(replicas.shard_columns(64, rank, ws))
        total = replicas.reduce_sum(len(mine), ws)
        gathered = [None] * ws
        dist.all_gather_object(gathered, mine)
        out[rank] = (t, total, sorted(c for g in gathered for c in g))
        replicas.barrier(ws)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_max_and_shard_union():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, total, union = res[rank]
        assert t == 2.5
        assert total == 64
        assert union == list(range(64))
