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


class _FakeImex:
    """Stand-in for the library in bench.measure_batched: a context records
    the source positions it was given and reports fixed counts."""

    class Imex:
        made = []

        def __init__(self, w, ncols):
            self.src = [tuple(p) for p in w.src_pos]
            self.ncols = ncols
            _FakeImex.Imex.made.append(self)

        @classmethod
        def from_workload(cls, w, ncols=1):
            return cls(w, ncols)

        def info(self):
            return {"n_d": 1000, "n_c": 24, "explicit_variant": 0, "explicit_tile_us_large": 1.0,
                    "explicit_tile_us_small": 0.0, "explicit_sweep_us": 0.0, "explicit_sweep_short_us": 0.0,
                    "explicit_split_us": [0.0] * 4, "solve_col_block": 1, "solve_col_block_us": [0.0] * 7}

        def step(self, n, stream=None):
            pass

        def close(self):
            pass


def _bench_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2310_14712_gb300 import workloads
        # Device time of a rank's steps: rank r takes (r + 1) ms for 10 steps.
        bench.time_flushed = lambda g, steps, stream, flush: float(rank + 1)
        line = bench.measure_batched(_FakeImex, workloads, 10, None, None, rank, world)
        made = _FakeImex.Imex.made[-1]
        out[rank] = (line, made.ncols, made.src)
    finally:
        dist.destroy_process_group()


def test_bench_batched_columns_split_between_gloo_ranks():
    # bench.py --gpus N: the 64 batched columns are split between the ranks
    # (contiguous blocks, each column once) and the value counts all of them
    # over the slowest rank's time (max over ranks).
    from paper_2310_14712_gb300 import workloads
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_bench_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    full = [tuple(p) for p in workloads.multisource(nsrc=64).src_pos]
    assert res[0][2] + res[1][2] == full
    assert [res[r][1] for r in range(world)] == [32, 32]
    for r in range(world):
        line = res[r][0]
        assert line["columns_per_rank"] == [32, 32]
        assert line["ncols"] == 64
        assert line["ms_per_step"] == 2.0 / 10          # the slower rank's time
        assert line["value"] == (1000 + 24) * 64 * 10 / (2.0e-3)
        assert "plain_value" not in line
