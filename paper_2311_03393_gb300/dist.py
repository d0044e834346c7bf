"""Host-side helpers for running independent replicas on several GPUs.

The discord-mining path shards by whole series (independent problems), so
ranks exchange nothing on the data path; only the timing (max over ranks) and
the totals (sum over ranks) are reduced, on the host.
"""
from __future__ import annotations

import os


def world() -> tuple:
    """(rank, local_rank, world_size) from the torchrun environment (1 process if unset)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def shard_by_cells(cells_per_series, world_size: int) -> list:
    """Assign series to ranks, largest first onto the least-loaded rank.

    Returns a list of index lists, one per rank.  Every series is assigned to
    exactly one rank; loads differ by at most the largest single series.
    """
    order = sorted(range(len(cells_per_series)), key=lambda i: (-cells_per_series[i], i))
    load = [0] * world_size
    out = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += cells_per_series[i]
    for r in range(world_size):
        out[r].sort()
    return out


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s replica workload (rank 0 keeps the base seed)."""
    return base if rank == 0 else base + 7919 * rank


def reduce_max_sum(value_max: float, value_sum: float, group=None) -> tuple:
    """(max over ranks of value_max, sum over ranks of value_sum) via torch.distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value_max, value_sum
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    a = torch.tensor([value_max], dtype=torch.float64, device=dev)
    b = torch.tensor([value_sum], dtype=torch.float64, device=dev)
    dist.all_reduce(a, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(b, op=dist.ReduceOp.SUM, group=group)
    return float(a.item()), float(b.item())
