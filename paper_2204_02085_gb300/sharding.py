"""Host-side bookkeeping for running the aligner on several GPUs.

Read pairs are independent (the paper aligns each pair on its own, with no
communication between processing units, Sec. I), so the multi-GPU form is
replicas: each rank aligns its own shard and no alignment data crosses
ranks.  The only collectives are bookkeeping ones: a barrier around the
timed region and the maximum of the ranks' elapsed times.
"""

from __future__ import annotations

import os


def dist_env() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [begin, end) share of n units for rank; shares differ by at
    most one unit and cover [0, n) exactly."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def shard_seed(seed: int, rank: int) -> int:
    """Seed of rank's own shard of a weak-scaling workload (rank 0 keeps the
    workload's seed)."""
    return seed if rank == 0 else seed + 7919 * rank


def max_over_ranks(value: float, group=None) -> float:
    """Maximum of a per-rank float across the process group (identity when
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def barrier(group=None) -> None:
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.barrier(group=group)
