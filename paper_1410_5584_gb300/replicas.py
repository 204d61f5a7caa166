"""Independent replicas, one process per GPU.

The fluctuating update of independent boxes needs no data exchange, so a
multi-GPU run is a set of replicas (distinct noise keys) and only the timing is
combined: the job time is the maximum over ranks and the work is the sum.
"""
from __future__ import annotations

MASK64 = (1 << 64) - 1


def replica_seed(base_seed: int, rank: int) -> int:
    """Distinct 64-bit Philox key per rank (a Weyl sequence over the ranks)."""
    return (int(base_seed) + 0x9E3779B97F4A7C15 * int(rank)) & MASK64


def aggregate(seconds: float, units: float, device=None):
    """(max seconds over ranks, sum of units over ranks); identity when
    torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(seconds), float(units)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
