"""CUDA-graph plans and the autotuner (through the C ABI)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_12349_b300 import binding as B
from paper_2507_12349_b300 import inputs as I

pytestmark = pytest.mark.gpu


def test_batch_plan_matches_direct_call_uneven_orders():
    w = I.WORKLOADS["su6_sym_uneven_n4_12"]
    cfgs = I.workload_configs(w, 1500)
    tabs = B.tables_for(w.model)
    d = B.configs_to_device(cfgs)
    ref = torch.empty(cfgs.n_cfg, dtype=torch.float64, device="cuda")
    B.cos_connected_sum_batch(tabs, 12, *d, "fp64", ref)
    B.cos_sync_status()
    out = torch.full_like(ref, float("nan"))
    plan = B.cos_plan_create_batch(tabs, 12, *d, "fp64", out)
    assert torch.equal(out, ref)                 # the eager sizing run
    out.fill_(float("nan"))
    for _ in range(2):
        plan.launch()
    plan.status()
    assert torch.equal(out, ref)
    assert plan.grid() >= 1
    # new inputs at the same addresses are picked up by the next replay
    L2 = w.model.L ** 2
    d[2].copy_((d[2] + 37) % L2)
    d[3].copy_(torch.remainder(d[3] + 0.37 * w.model.beta, w.model.beta))
    ref2 = torch.empty_like(ref)
    B.cos_connected_sum_batch(tabs, 12, *d, "fp64", ref2)
    plan.launch()
    plan.status()
    assert torch.equal(out, ref2)
    plan.close()
    tabs.close()


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_matrices_plan_with_shifts_and_mass(prec):
    n, n_mat, ncfg = 7, 3, 100
    Ms = I.random_matrices(3, ncfg, n_mat, n, 0.9)
    order = torch.full((ncfg,), n, dtype=torch.int32, device="cuda")
    moff = torch.arange(ncfg, dtype=torch.int64, device="cuda") * n_mat * n * n
    M = torch.tensor(Ms.ravel(), device="cuda")
    sig = [0.1, -0.2, 0.05]
    ref, refm = (torch.empty(ncfg, dtype=torch.float64, device="cuda") for _ in range(2))
    B.cos_connected_sum_matrices(n, order, moff, n_mat, 1, sig, M, prec, ref, refm)
    out, mass = (torch.empty_like(ref) for _ in range(2))
    plan = B.cos_plan_create_matrices(n, order, moff, n_mat, 1, sig, M, prec, out, mass)
    out.zero_(); mass.zero_()
    plan.launch()
    plan.status()
    assert torch.equal(out, ref) and torch.equal(mass, refm)
    plan.close()


def test_plan_reports_device_status():
    order = torch.tensor([4, 9, 4], dtype=torch.int32, device="cuda")   # 9 > n_max
    moff = torch.arange(3, dtype=torch.int64, device="cuda") * 16
    M = torch.tensor(I.random_matrices(1, 3, 1, 4).ravel(), device="cuda")
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    plan = B.cos_plan_create_matrices(4, order, moff, 1, 2, None, M, "fp64", out)
    with pytest.raises(B.CosError) as ei:
        plan.status()                  # the eager run flagged the order
    assert ei.value.status == -2
    plan.launch()
    with pytest.raises(B.CosError):
        plan.status()                  # and so does every replay
    plan.close()


def test_autotune_installs_a_shape_and_keeps_results():
    n, n_mat = 6, 2
    Ms = I.random_matrices(8, 300, n_mat, n, 0.9)
    order = torch.full((300,), n, dtype=torch.int32, device="cuda")
    moff = torch.arange(300, dtype=torch.int64, device="cuda") * n_mat * n * n
    M = torch.tensor(Ms.ravel(), device="cuda")
    ref = torch.empty(300, dtype=torch.float64, device="cuda")
    B.cos_connected_sum_matrices(n, order, moff, n_mat, 1, None, M, "fp64", ref)
    w, c, pf, ms = B.cos_autotune(n, n_mat, 1, False, "fp64", 2000)
    assert 1 <= w <= 16 and 1 <= c <= 8 and ms > 0
    assert B.cos_get_tuning(n, "fp64", n_mat) == (w, c, pf)
    out = torch.empty_like(ref)
    B.cos_connected_sum_matrices(n, order, moff, n_mat, 1, None, M, "fp64", out)
    B.cos_sync_status()
    assert torch.equal(out, ref)     # per-lane arithmetic does not depend on the launch shape
    B.cos_set_tuning(n, "fp64", n_mat, 8, 2, 1)


def test_release_workspace_frees_and_recreates():
    """cos_release_workspace returns the stream's cached workspace to the device; the next call
    allocates a fresh one and gives the same bits."""
    import numpy as np
    n, n_mat, ncfg = 8, 2, 64
    Ms = I.random_matrices(5, ncfg, n_mat, n, 0.9)
    order = torch.full((ncfg,), n, dtype=torch.int32, device="cuda")
    moff = torch.arange(ncfg, dtype=torch.int64, device="cuda") * n_mat * n * n
    M = torch.tensor(Ms, device="cuda").contiguous()
    out1 = torch.empty(ncfg, dtype=torch.float64, device="cuda")
    out2 = torch.empty_like(out1)
    B.cos_connected_sum_matrices(n, order, moff, n_mat, 1, None, M, "fp64", out1)
    B.cos_sync_status()
    free_before = torch.cuda.mem_get_info()[0]
    B.cos_release_workspace()
    assert torch.cuda.mem_get_info()[0] > free_before          # the layer ring went back to the device
    B.cos_connected_sum_matrices(n, order, moff, n_mat, 1, None, M, "fp64", out2)
    B.cos_sync_status()
    assert np.array_equal(out1.cpu().numpy(), out2.cpu().numpy())


@pytest.mark.parametrize("prec,n,n_mat", [("mixed", 8, 4), ("mixed", 10, 3), ("df64", 8, 4), ("df64", 9, 2)])
def test_prefetch_modes_leave_results_bitwise(prec, n, n_mat):
    """Prefetch modes 0-4 of the pair kernels (none, next mask into L2 or L1, next row into L1,
    both) and the launch shapes only move data: the connected sums are bit for bit the same,
    with shifts and an uneven tail of orders."""
    ncfg = 300
    orders = np.array([n - (c % 3 == 2) for c in range(ncfg)], dtype=np.int32)
    Ms = [I.random_matrices(77 + c, 1, n_mat, int(orders[c]), 0.9)[0] for c in range(ncfg)]
    moff = np.concatenate([[0], np.cumsum([m.size for m in Ms])[:-1]]).astype(np.int64)
    d_order = torch.tensor(orders, device="cuda")
    d_moff = torch.tensor(moff, device="cuda")
    M = torch.tensor(np.concatenate([m.ravel() for m in Ms]), device="cuda")
    sigma = list(np.linspace(-0.1, 0.12, n_mat))
    saved = B.cos_get_tuning(n, prec, n_mat)
    outs = []
    try:
        for w, c, pf in [(16, 1, 0), (16, 1, 1), (16, 1, 2), (16, 1, 3), (16, 1, 4), (8, 1, 3)]:
            B.cos_set_tuning(n, prec, n_mat, w, c, pf)
            out = torch.empty(ncfg, dtype=torch.float64, device="cuda")
            B.cos_connected_sum_matrices(n, d_order, d_moff, n_mat, 1, sigma, M, prec, out)
            B.cos_sync_status()
            outs.append(out.cpu().numpy())
    finally:
        B.cos_set_tuning(n, prec, n_mat, *saved)
    assert np.all(np.isfinite(outs[0]))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
