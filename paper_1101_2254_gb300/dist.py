"""Host-side bookkeeping of runs over several GPUs, one process per GPU.

Stamps are independent, so the fitting path has no exchange step and needs no
collective on its data: each rank fits its own stamps (weak scaling).  The only
collectives are a barrier before the timed region and the maximum over ranks of
the timed milliseconds, so that the slowest rank sets the reported time.
Ranks are launched by torchrun (RANK, LOCAL_RANK, WORLD_SIZE, MASTER_*); with
no GPU the gloo backend serves the same calls.
"""
from __future__ import annotations

import os


def env():
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(world: int):
    import torch
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")


def finalize(world: int):
    import torch.distributed as dist
    if world > 1 and dist.is_initialized():
        dist.destroy_process_group()


def shard(count: int, rank: int, world: int):
    """Contiguous [start, stop) share of `count` units for `rank`: sizes differ by at most one."""
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def barrier(world: int):
    import torch.distributed as dist
    if world > 1:
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The largest `x` over the ranks (every rank gets it)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
