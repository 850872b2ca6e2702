"""Host logic of the multi-process form: one process per GPU, no data-path
collective.  The method's independent problems (replicas of a workload, or
the source columns of a batched workload) are split across ranks; timing
takes the maximum over ranks.  Works with any torch.distributed backend
(nccl on GPUs, gloo in the CPU tests)."""
import os


def dist_env():
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_columns(ncols, rank, world):
    """Contiguous block of source columns for `rank`: sizes differ by at most
    one, lower ranks take the larger blocks, every column exactly once."""
    if world < 1 or not 0 <= rank < world or ncols < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(ncols, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def reduce_max(x, world, device=None):
    """Maximum of a float over the ranks (identity for one process)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x, world, device=None):
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
