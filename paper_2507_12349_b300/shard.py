"""Sharding of Monte Carlo configurations over ranks (one process per GPU).

Configurations are independent samples, so the hot path needs no collective:
each rank evaluates its own configurations, and the only exchange is one
all-reduce of per-order accumulators (sum of c, sum of c^2, count) at the end,
a few hundred bytes.
"""
from __future__ import annotations

import numpy as np

N_ORDERS = 13  # orders 0..12


def shard_bounds(n_total: int, rank: int, world: int):
    """Contiguous near-equal block [start, stop) of rank `rank` among `world`."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def per_order_accumulators(order: np.ndarray, values: np.ndarray) -> np.ndarray:
    """[N_ORDERS][3] float64: per order, sum of values, sum of squares, count."""
    order = np.asarray(order, dtype=np.int64)
    values = np.asarray(values, dtype=np.float64)
    acc = np.zeros((N_ORDERS, 3), dtype=np.float64)
    np.add.at(acc[:, 0], order, values)
    np.add.at(acc[:, 1], order, values * values)
    np.add.at(acc[:, 2], order, 1.0)
    return acc


def allreduce_accumulators(acc: np.ndarray, device: str = "cpu") -> np.ndarray:
    """Sum the accumulators of every rank (torch.distributed, already initialized)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(acc, dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()
