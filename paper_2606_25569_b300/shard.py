"""Sharding of a suspension over ranks (one process per GPU): host logic only.

The per-vesicle work of a step is independent across vesicles, so ranks own contiguous ranges of
vesicles; the far field is the one exchange: every rank needs every source point (its FP32 source
record and centre) and evaluates the sum for its own targets. `partition` balances the ranges,
`allgather_rows` is that exchange (any torch.distributed backend: NCCL between GPUs, gloo on the
host), and `job_throughput` is the whole-job figure of a timed region (slowest rank, all units).
"""
import numpy as np


def partition(counts, world, weights=None):
    """Contiguous vesicle ranges [(v0, v1)] per rank, balancing sum(weights) (default N_v^2, the
    per-vesicle dense algebra; the far field's share N_v * P is proportional to N_v); every rank gets
    at least one vesicle when there are enough."""
    counts = np.asarray(counts, dtype=np.int64)
    M = len(counts)
    if world < 1:
        raise ValueError("world must be >= 1")
    w = counts.astype(np.float64) ** 2 if weights is None else np.asarray(weights, dtype=np.float64)
    cum = np.concatenate([[0.0], np.cumsum(w)])
    total = cum[-1]
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        v = int(np.searchsorted(cum, target, side="left"))
        # nearest boundary to the target, kept increasing and leaving room for the later ranks
        if v > 0 and abs(cum[v - 1] - target) <= abs(cum[min(v, M)] - target):
            v -= 1
        v = max(v, bounds[-1] + (1 if bounds[-1] < M else 0))
        v = min(v, M - (world - r) if M >= world else M)
        bounds.append(v)
    bounds.append(M)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def allgather_rows(t, group=None):
    """Concatenate, in rank order, every rank's tensor t (same trailing shape, any number of rows)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = torch.tensor([t.shape[0]], dtype=torch.int64, device=t.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    m = max(sizes)
    pad = torch.zeros((m,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
    pad[:t.shape[0]] = t
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:s] for p, s in zip(parts, sizes)])


def job_throughput(units_local, ms_local, group=None):
    """(units of all ranks / slowest rank's seconds, slowest rank's ms) of one timed region."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return units_local / (ms_local * 1e-3), ms_local
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    ms = torch.tensor([float(ms_local)], dtype=torch.float64, device=dev)
    units = torch.tensor([float(units_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(ms, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(units, op=dist.ReduceOp.SUM, group=group)
    return float(units.item()) / (float(ms.item()) * 1e-3), float(ms.item())
