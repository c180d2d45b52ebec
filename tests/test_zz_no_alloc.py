"""The allocation-free entry point against the regular one.

cos_connected_sum_matrices_noalloc serves callers that may not allocate device
memory (an allocator-less plug-in, a process whose device memory belongs to a
pool): its scratch lives in a fixed static device array.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it passes on its own in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_12349_b300 import binding as B
from paper_2507_12349_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _call(fn, order, moff, n_mat, wt, sigma, M, prec, out, mass):
    lib = B.lib()
    sig = None if sigma is None else (ctypes.c_double * n_mat)(*sigma)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, fn)(int(order.numel()), int(order.max().item()), ctypes.c_void_p(order.data_ptr()),
                          ctypes.c_void_p(moff.data_ptr()), n_mat, wt, sig, ctypes.c_void_p(M.data_ptr()),
                          B.PRECISIONS[prec], ctypes.c_void_p(out.data_ptr()),
                          ctypes.c_void_p(mass.data_ptr() if mass is not None else 0), stream)
    assert rc == 0, (fn, rc, lib.cos_last_error())


def _case(seed, ncfg, n_mat, orders):
    rng = np.random.default_rng(seed)
    order = rng.choice(orders, size=ncfg).astype(np.int32)
    Ms = [I.random_matrices(seed * 1000 + c, 1, n_mat, int(n), 0.9)[0] for c, n in enumerate(order)]
    moff = B.matrix_offsets(order, n_mat)
    flat = np.concatenate([m.ravel() for m in Ms])
    return (torch.tensor(order, device="cuda"), torch.tensor(moff, device="cuda"), torch.tensor(flat, device="cuda"))


@pytest.mark.parametrize("prec", ["fp64", "mixed", "df64"])
def test_noalloc_matches_regular_entry_on_two_calls(prec):
    calls = [  # (seed, configurations, matrices per configuration, loop weight, sigma, orders)
        (11, 77, 3, 1, [0.1, 0.0, -0.08], [5, 7, 8]),
        (12, 130, 1, 4, None, [3, 6, 9, 10]),
    ]
    for seed, ncfg, n_mat, wt, sigma, orders in calls:
        order, moff, M = _case(seed, ncfg, n_mat, orders)
        ref = torch.empty(ncfg, dtype=torch.float64, device="cuda")
        ref_mass = torch.empty_like(ref)
        got = torch.empty_like(ref)
        got_mass = torch.empty_like(ref)
        _call("cos_connected_sum_matrices", order, moff, n_mat, wt, sigma, M, prec, ref, ref_mass)
        B.cos_sync_status()
        _call("cos_connected_sum_matrices_noalloc", order, moff, n_mat, wt, sigma, M, prec, got, got_mass)
        torch.cuda.synchronize()
        r, g, m = ref.cpu().numpy(), got.cpu().numpy(), ref_mass.cpu().numpy()
        n = order.cpu().numpy()
        # same tolerance as the parity tests, stated against the absolute mass
        if prec == "df64":
            tol = (16 * n * n + 64 * n) * 2.0 ** -48 * m
        else:
            tol = 64 * n * (2.0 ** -53 if prec == "fp64" else 2.0 ** -24) * m
        assert np.all(np.isfinite(g))
        assert np.all(np.abs(g - r) <= tol)
        assert np.allclose(got_mass.cpu().numpy(), m, rtol=1e-12)


def test_noalloc_rejects_orders_beyond_its_workspace():
    order = torch.tensor([11], dtype=torch.int32, device="cuda")
    moff = torch.zeros(1, dtype=torch.int64, device="cuda")
    M = torch.zeros(121, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(B.CosError) as ei:
        B.cos_connected_sum_matrices_noalloc(11, order, moff, 1, 2, None, M, "fp64", out)
    assert ei.value.status == -2


def test_noalloc_order_above_n_max_stays_nan():
    """A configuration whose order exceeds n_max is skipped by the planner and keeps the NaN
    the call writes first; the others are computed as usual."""
    order, moff, M = _case(21, 40, 2, [4, 6])
    order[7] = 7                                   # above n_max = 6; its matrices are never read
    out = torch.zeros(40, dtype=torch.float64, device="cuda")
    ref = torch.zeros_like(out)
    keep = torch.ones(40, dtype=torch.bool)
    keep[7] = False
    B.cos_connected_sum_matrices_noalloc(6, order, moff, 2, 1, None, M, "fp64", out)
    torch.cuda.synchronize()
    sub = torch.arange(40, device="cuda")[keep.cuda()]
    ref_sub = torch.zeros(len(sub), dtype=torch.float64, device="cuda")
    B.cos_connected_sum_matrices(6, order[sub].contiguous(), moff[sub].contiguous(), 2, 1, None, M, "fp64", ref_sub)
    B.cos_sync_status()
    got = out.cpu().numpy()
    assert np.isnan(got[7])
    assert np.array_equal(got[keep.numpy()], ref_sub.cpu().numpy())


def test_noalloc_rejects_batch_too_large_for_the_array():
    """At n_max = 10 one FP64 layer ring takes about 59 MB of the 128 MiB array; 20 million
    configurations need another 90 MB of batch tables, so the call returns COS_ERR_ARG
    before launching anything.  (The buffers are sized so that every access of a launch
    would stay in bounds even if the check were missing.)"""
    ncfg = 20_000_000
    order = torch.full((ncfg,), 10, dtype=torch.int32, device="cuda")
    moff = torch.zeros(ncfg, dtype=torch.int64, device="cuda")
    M = torch.full((100,), 0.1, dtype=torch.float64, device="cuda")
    out = torch.zeros(ncfg, dtype=torch.float64, device="cuda")
    with pytest.raises(B.CosError) as ei:
        B.cos_connected_sum_matrices_noalloc(10, order, moff, 1, 2, None, M, "fp64", out)
    assert ei.value.status == -1
    assert "too large" in str(ei.value)
    torch.cuda.synchronize()
    assert float(out.abs().max().item()) == 0.0    # nothing was written


_FRESH_PROCESS = r"""
import os, sys, numpy as np, torch
sys.path.insert(0, os.environ["COS_REPO_ROOT"])
from paper_2507_12349_b300 import binding as B
B.lib()
torch.cuda.init()
n_cfg, n = 64, 8
order = torch.full((n_cfg,), n, dtype=torch.int32, device="cuda")
moff = torch.arange(n_cfg, dtype=torch.int64, device="cuda") * n * n
M = torch.rand(n_cfg * n * n, dtype=torch.float64, device="cuda", generator=None) * 0.4
out = torch.empty(n_cfg, dtype=torch.float64, device="cuda")
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
B.cos_connected_sum_matrices_noalloc(n, order, moff, 1, 2, None, M, "fp64", out)
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
for _ in range(5):
    B.cos_connected_sum_matrices_noalloc(n, order, moff, 1, 2, None, M, "fp64", out)
torch.cuda.synchronize()
free2 = torch.cuda.mem_get_info()[0]
print(free0, free1, free2)
"""


def test_noalloc_first_call_takes_the_array_and_later_calls_allocate_nothing():
    """In a fresh process under lazy module loading: free device memory drops by the 128 MiB
    array (plus a little kernel code) at the first call, and not at all over five more."""
    import os
    import subprocess
    import sys
    env = dict(os.environ, CUDA_MODULE_LOADING="LAZY",
               COS_REPO_ROOT=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    r = subprocess.run([sys.executable, "-c", _FRESH_PROCESS], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    free0, free1, free2 = (int(x) for x in r.stdout.split()[-3:])
    mib = 1 << 20
    assert 128 * mib <= free0 - free1 <= 192 * mib, (free0, free1)
    assert free2 == free1
