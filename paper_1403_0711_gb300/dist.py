"""Host-side combination across processes (one process per GPU).

Chains are independent, so N GPUs run N replicas and the only exchange is at
the end: the per-chain estimator rows of every rank are gathered in rank
order and pooled with coulps_pool_stats (the counterpart of the paper's final
mpi_reduce), and benchmark timings take the maximum over ranks.  Works with
any torch.distributed backend (NCCL between GPUs, gloo on CPU).
"""
from __future__ import annotations

import numpy as np

from . import coulps


def _dist():
    import torch.distributed as dist
    return dist


def _device():
    import torch
    dist = _dist()
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def max_over_ranks(value: float) -> float:
    import torch
    dist = _dist()
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(rows: np.ndarray) -> np.ndarray:
    """Concatenate every rank's (n_k, STAT_STRIDE) rows in rank order."""
    import torch
    dist = _dist()
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.float64).reshape(-1, coulps.STAT_STRIDE))
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return rows
    dev = _device()
    n = torch.tensor([len(rows)], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(n) for _ in range(dist.get_world_size())]
    dist.all_gather(counts, n)
    m = int(max(int(c.item()) for c in counts))
    buf = torch.zeros((m, coulps.STAT_STRIDE), dtype=torch.float64, device=dev)
    buf[: len(rows)] = torch.from_numpy(rows).to(dev)
    parts = [torch.zeros_like(buf) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, buf)
    return np.concatenate([p[: int(c.item())].cpu().numpy() for p, c in zip(parts, counts)])


def pooled_estimate(rows: np.ndarray) -> dict:
    """Pooled estimate over all ranks' chains (every rank gets the result)."""
    return coulps.pool_stats(gather_rows(rows))
