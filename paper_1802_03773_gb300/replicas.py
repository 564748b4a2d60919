"""Host-side helpers for running independent problems on several GPUs (one process per GPU).

The hot path has no exchange step between ranks: every rank solves its own problems (its own
seed offset, or its own contiguous share of a batch) and only the timing is combined, as the
maximum over ranks.  These helpers work with any torch.distributed backend (NCCL on GPUs,
gloo on CPU for tests).
"""
from __future__ import annotations

import os


def dist_env():
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def share(total: int, rank: int, world: int):
    """Contiguous share [lo, hi) of `total` independent units for `rank` of `world`; the shares
    cover every unit exactly once and differ in size by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    base, extra = divmod(int(total), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of `value` over the ranks of the default process group (value itself when
    no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
