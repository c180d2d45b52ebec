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


def weak_block(n_per_rank: int, rank: int):
    """Weak scaling: rank r takes configurations [r n, (r + 1) n) of the seeded stream, so the
    work per GPU is fixed as ranks are added (the benchmark's multi-GPU layout)."""
    if n_per_rank < 0 or rank < 0:
        raise ValueError("bad shard arguments")
    return rank * n_per_rank, (rank + 1) * n_per_rank


def sharded_accumulators(order: np.ndarray, compute, rank: int, world: int, device: str = "cpu") -> np.ndarray:
    """The multi-GPU form of an MC estimate: this rank's contiguous block of the configurations
    (`order` holds every configuration's order), evaluated by `compute(start, stop)` -> the
    connected sums of configurations start .. stop - 1 (on this rank's GPU: the batch call on
    that slice), reduced to per-order accumulators and summed over ranks with one all-reduce.
    Returns the global [N_ORDERS][3] accumulators on every rank."""
    start, stop = shard_bounds(len(order), rank, world)
    vals = np.asarray(compute(start, stop), dtype=np.float64) if stop > start else np.zeros(0)
    return allreduce_accumulators(per_order_accumulators(np.asarray(order)[start:stop], vals), device)


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
