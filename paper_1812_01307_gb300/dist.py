"""Multi-process helpers for running independent reconstructions on several
GPUs of one node (one process per GPU).

BSGD-TV's data-parallel form here is weak scaling over independent problems
(slices of a volume share nothing), so ranks exchange no data on the hot
path: only a barrier and a max-over-ranks of the elapsed time, as the
timing contract requires.
"""
from __future__ import annotations

import os


def env_rank():
    """(rank, local_rank, world_size) from the torchrun environment (0, 0, 1 if absent)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def shard(n_items: int, rank: int, world: int):
    """Contiguous share [start, stop) of n_items for `rank` (array_split rule)."""
    q, rem = divmod(n_items, world)
    start = rank * q + min(rank, rem)
    return start, start + q + (1 if rank < rem else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group (identity if
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
