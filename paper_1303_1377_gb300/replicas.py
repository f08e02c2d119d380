"""Independent replicas on several GPUs (one process per GPU).

The two-level solve of one lattice does not shard across GPUs in this library
(the method's domain decomposition over processes is not built), so N GPUs run N
independent replicas of the workload: every rank solves its own batch of
right-hand sides with its own handle, and the only communication is the timing
aggregate below (no data-path collective).
"""
from __future__ import annotations


def rhs_slice(n_total: int, rank: int, world: int) -> range:
    """Right-hand sides of an n_total batch handled by `rank` when one batch is spread
    over `world` replicas (contiguous, sizes differ by at most one)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def aggregate(ms_local: float, units_local: float, dist=None, device=None):
    """Whole-job throughput: units summed over ranks / slowest rank's time (ms).

    Returns (units_per_second, max_ms, total_units).  With dist=None (one process)
    the local values are used."""
    if dist is None:
        return units_local / (ms_local / 1e3), ms_local, units_local
    import torch

    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / (float(t.item()) / 1e3), float(t.item()), float(u.item())
