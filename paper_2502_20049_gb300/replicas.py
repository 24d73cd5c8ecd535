"""Rank bookkeeping for running independent replicas on several GPUs.

The PSM path has no data-path collective on one node in this library: every
rank runs its own replica of a workload (weak scaling).  Only the timing needs
the ranks: a barrier around the timed region and the maximum time over ranks.
"""

from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the torchrun environment (defaults 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str | None = None, timeout_s: float | None = None):
    """Initialise torch.distributed when WORLD_SIZE > 1; returns the module or None.

    timeout_s bounds every collective: a rank that left (raised, exited) makes
    the others' next barrier or reduction fail with an error after at most
    that long instead of waiting forever (None: torch's default)."""
    rank, world, _ = env()
    if world <= 1:
        return None
    import datetime

    import torch
    import torch.distributed as dist

    if not dist.is_initialized():
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        kw = {} if timeout_s is None else {"timeout": datetime.timedelta(seconds=timeout_s)}
        dist.init_process_group(backend, **kw)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float, device=None) -> float:
    """Maximum of a float over all ranks (the value itself with one rank)."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, t_max: float) -> float:
    """Whole-job throughput: the units all ranks processed / the slowest rank's time."""
    return units_per_rank * world / t_max
