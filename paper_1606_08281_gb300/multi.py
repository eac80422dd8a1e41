"""Multi-GPU data parallelism for the likelihood batches (replicas).

Filters are independent and the only reduction (over the trajectories of one
theta) stays on one GPU, so ranks never exchange data on the compute path:
each rank evaluates its own batch of theta rows (weak scaling).  The only
collectives are host-side bookkeeping: a barrier around the timed region and
the maximum of the ranks' times, and (for a sharded batch) gathering the
per-rank log-likelihoods.
"""
from __future__ import annotations

import numpy as np

from . import workloads as W


def rank_thetas(w: W.Workload, rank: int) -> np.ndarray:
    """Rank 0 evaluates the workload's own theta batch; rank r > 0 draws an
    independent batch of the same size from the same prior (seed offset)."""
    if rank == 0:
        return w.thetas()
    rng = np.random.default_rng(w.theta_seed + 7919 * rank)
    return np.ascontiguousarray(W.log_uniform(rng, w.prior_lo, w.prior_hi, w.M))


def shard_rows(M: int, rank: int, world: int) -> slice:
    """Contiguous theta-row range of `rank` when one batch is split over ranks."""
    base, extra = divmod(M, world)
    start = rank * base + min(rank, extra)
    return slice(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(local: np.ndarray, M: int, device=None) -> np.ndarray:
    """Concatenate per-rank results of a batch split by shard_rows (rank order)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return np.asarray(local)
    world = dist.get_world_size()
    sizes = [shard_rows(M, r, world).stop - shard_rows(M, r, world).start for r in range(world)]
    width = max(sizes)
    buf = torch.full((width,), float("nan"), dtype=torch.float64, device=device)
    buf[: len(local)] = torch.as_tensor(np.asarray(local), dtype=torch.float64)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    return np.concatenate([p[:n].cpu().numpy() for p, n in zip(parts, sizes)])
