"""The multi-rank path on CPU: two gloo ranks shard configurations, evaluate them
(here with the CPU oracle, standing in for one GPU each) and all-reduce the
per-order accumulators; the result equals the single-process total."""
import os
import socket

import numpy as np
import pytest

from paper_2507_12349_b300 import shard as S


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _values(order, first=0):
    """Connected sums of configurations first, first+1, ... (matrices seeded by global index)."""
    import oracle as O
    from paper_2507_12349_b300 import inputs as I
    out = []
    for c, n in enumerate(order):
        M = I.random_matrices(900 + first + c, 1, 1, int(n), 0.8)[0]
        out.append(O.dp(M, None, weight=3))
    return np.array(out)


def _worker(rank, world, port, order, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start, stop = S.shard_bounds(len(order), rank, world)
    # the oracle stands in for the GPU batch call on this rank's slice
    tot = S.sharded_accumulators(order, lambda a, b: _values(order[a:b], first=a), rank, world)
    q.put((rank, start, stop, tot))
    dist.barrier()
    dist.destroy_process_group()


def test_weak_blocks_tile_the_stream():
    assert [S.weak_block(5, r) for r in range(3)] == [(0, 5), (5, 10), (10, 15)]
    with pytest.raises(ValueError):
        S.weak_block(-1, 0)


def test_shard_bounds_partition():
    for n in (0, 1, 7, 100):
        for world in (1, 2, 3, 8):
            spans = [S.shard_bounds(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1


def test_two_gloo_ranks_allreduce_per_order_sums():
    import torch.multiprocessing as mp
    rng = np.random.default_rng(0)
    order = rng.integers(2, 6, size=23)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, order, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full = S.per_order_accumulators(order, _values(order))
    for _, _, _, tot in res:
        assert np.allclose(tot, full, rtol=1e-13, atol=0)
    spans = sorted((r[1], r[2]) for r in res)
    assert spans[0][0] == 0 and spans[1][1] == len(order) and spans[0][1] == spans[1][0]
