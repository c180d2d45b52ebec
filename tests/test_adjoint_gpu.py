"""GPU parity of the adjoint DP (through the C ABI) against the oracle.

References:
  * dc/dM: central differences of the __float128 oracle DP.  c is a quadratic
    polynomial in every single entry (a vertex has two points, so a cover uses an
    entry at most twice; pinned in test_oracle_pins), so the central difference
    with any step is exact up to rounding.
  * dc/dsigma: exact derivative of a polynomial fit in sigma (degree <= n).
  * dense autograd through the torch brute-force sum for n <= 3.
  * dc/dmu, dc/dalpha through the tables: central differences of the oracle
    pipeline (tables rebuilt, gathered, DP) with step 1e-6 in FP64.
Tolerance: |err| <= 1e-9 * (|ref| + scale), scale = the largest reference entry.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from oracle import propagators as P
from paper_2507_12349_b300 import autograd as AG
from paper_2507_12349_b300 import binding as B
from paper_2507_12349_b300 import inputs as I

pytestmark = pytest.mark.gpu


def pack(Ms, n_mat):
    order = np.array([m.shape[-1] for m in Ms], dtype=np.int32)
    moff = B.matrix_offsets(order, n_mat)
    flat = np.concatenate([np.asarray(m).ravel() for m in Ms])
    return (torch.tensor(order, device="cuda"), torch.tensor(moff, device="cuda"),
            torch.tensor(flat, device="cuda"), order, moff)


def gpu_grad(Ms, n_mat, wt, sigma, gout):
    d_order, d_moff, d_M, order, moff = pack(Ms, n_mat)
    n = len(Ms)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    gM = torch.full_like(d_M, float("nan"))
    gs = torch.full((n, n_mat), float("nan"), dtype=torch.float64, device="cuda")
    B.cos_connected_sum_matrices_grad(int(order.max()), d_order, d_moff, n_mat, wt, sigma, d_M,
                                      torch.tensor(gout, dtype=torch.float64, device="cuda"), out, gM, gs)
    B.cos_sync_status()
    g = gM.cpu().numpy()
    return out.cpu().numpy(), [g[moff[c]:moff[c] + Ms[c].size].reshape(Ms[c].shape) for c in range(n)], gs.cpu().numpy()


def exact_dM(M, sigma, wt, h=0.25):
    g = np.zeros_like(M)
    for idx in np.ndindex(*M.shape):
        Mp = M.copy(); Mp[idx] += h
        Mm = M.copy(); Mm[idx] -= h
        g[idx] = (O.dp(Mp, sigma, weight=wt, prec="q") - O.dp(Mm, sigma, weight=wt, prec="q")) / (2 * h)
    return g


def exact_dsigma(M, sigma, wt):
    n = M.shape[-1]
    s0 = np.zeros(M.shape[0]) if sigma is None else np.array(sigma, dtype=np.float64)
    out = []
    for l in range(len(s0)):
        hs = [0.05 * k for k in range(-n - 1, n + 2)]
        vals = []
        for h in hs:
            s2 = s0.copy(); s2[l] += h
            vals.append(O.dp(M, list(s2), weight=wt, prec="q"))
        out.append(np.polyfit(hs, vals, n + 1)[-2])
    return np.array(out)


def close(a, b, rel=1e-9):
    scale = max(np.max(np.abs(b)), 1e-300)
    return np.all(np.abs(a - b) <= rel * (np.abs(b) + scale))


@pytest.mark.parametrize("n,n_mat,wt,shifts,ncfg", [
    (1, 3, 1, True, 5), (2, 1, 4, False, 9), (3, 2, 1, True, 11), (4, 3, 1, False, 13), (4, 1, 6, True, 7),
    (5, 4, 1, False, 10), (5, 2, 1, True, 9),
])
def test_grad_matrices_vs_exact_differences(n, n_mat, wt, shifts, ncfg):
    Ms = list(I.random_matrices(500 + n * 10 + n_mat, ncfg, n_mat, n, 0.9))
    sigma = list(np.linspace(-0.15, 0.2, n_mat)) if shifts else None
    gout = np.linspace(0.5, 1.5, ncfg)
    out, gM, gs = gpu_grad(Ms, n_mat, wt, sigma, gout)
    for c in [0, ncfg // 2, ncfg - 1]:
        ref = O.dp(Ms[c], sigma, weight=wt, prec="ld")
        assert abs(out[c] - ref) <= 1e-12 * O.dp(Ms[c], sigma, weight=wt, absmode=True)
        assert close(gM[c], gout[c] * exact_dM(Ms[c], sigma, wt)), c
        assert close(gs[c], gout[c] * exact_dsigma(Ms[c], sigma, wt), rel=1e-7), c


def test_grad_matches_autograd_of_dense_brute_force():
    for n, n_mat, shifts in [(2, 2, True), (3, 2, False), (3, 3, True)]:
        M = I.random_matrices(42 + n, 1, n_mat, n, 0.9)[0]
        sigma = list(np.linspace(-0.2, 0.1, n_mat)) if shifts else None
        Mt = torch.tensor(M, requires_grad=True)
        st = torch.tensor(sigma, requires_grad=True) if shifts else None
        O.torch_brute(Mt, st).backward()
        _, gM, gs = gpu_grad([M], n_mat, 1, sigma, [1.0])
        assert close(gM[0], Mt.grad.numpy())
        if shifts:
            assert close(gs[0], st.grad.numpy())


def test_autograd_function_matrices():
    n, n_mat = 4, 3
    Ms = list(I.random_matrices(7, 6, n_mat, n, 0.9))
    d_order, d_moff, d_M, order, moff = pack(Ms, n_mat)
    M = d_M.clone().requires_grad_(True)
    sig = torch.tensor([0.1, -0.05, 0.2], dtype=torch.float64, requires_grad=True)
    c = AG.connected_sum(M, sig, d_order, d_moff, n, n_mat)
    w = torch.linspace(1.0, 2.0, 6, dtype=torch.float64, device="cuda")
    (c * w).sum().backward()
    g = M.grad.cpu().numpy()
    for k in (0, 5):
        ref = float(w[k]) * exact_dM(Ms[k], sig.tolist(), 1)
        assert close(g[moff[k]:moff[k] + Ms[k].size].reshape(Ms[k].shape), ref)
    ref_s = sum(float(w[k]) * exact_dsigma(Ms[k], sig.tolist(), 1) for k in range(6))
    assert close(sig.grad.numpy(), ref_s, rel=1e-7)


def test_grad_forward_value_and_determinism():
    Ms = list(I.random_matrices(3, 40, 4, 7, 0.9))
    d_order, d_moff, d_M, order, _ = pack(Ms, 4)
    ref = torch.empty(40, dtype=torch.float64, device="cuda")
    B.cos_connected_sum_matrices(7, d_order, d_moff, 4, 1, None, d_M, "fp64", ref)
    outs, gms = [], []
    for _ in range(2):
        out = torch.empty(40, dtype=torch.float64, device="cuda")
        gM = torch.empty_like(d_M)
        B.cos_connected_sum_matrices_grad(7, d_order, d_moff, 4, 1, None, d_M,
                                          torch.ones(40, dtype=torch.float64, device="cuda"), out, gM)
        outs.append(out.cpu().numpy())
        gms.append(gM.cpu().numpy())
    B.cos_sync_status()
    assert np.array_equal(outs[0], ref.cpu().numpy())      # same per-lane arithmetic as the forward kernel
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(gms[0], gms[1])


def test_grad_orders_11_12_euler_and_transpose():
    """Orders 11 and 12 (the 12-warp adjoint, every layer of order 12 kept: 2.2 GB per CTA),
    checked by properties that hold at any size: c is homogeneous of degree 2n in (M, sigma),
    so sum M dc/dM + sum sigma dc/dsigma = 2n c (Euler); transposing every matrix leaves c
    unchanged and transposes dc/dM; the forward value equals the forward kernel's bit for bit."""
    orders = [12, 11, 11, 12]
    n_mat = 2
    sigma = [0.07, -0.05]
    Ms = [I.random_matrices(1200 + c, 1, n_mat, n, 0.9)[0] for c, n in enumerate(orders)]
    gout = np.ones(len(Ms))
    out, gM, gs = gpu_grad(Ms, n_mat, 1, sigma, gout)
    outT, gMT, gsT = gpu_grad([np.ascontiguousarray(np.swapaxes(M, 1, 2)) for M in Ms], n_mat, 1, sigma, gout)
    d_order, d_moff, d_M, order, _ = pack(Ms, n_mat)
    ref = torch.empty(len(Ms), dtype=torch.float64, device="cuda")
    B.cos_connected_sum_matrices(12, d_order, d_moff, n_mat, 1, sigma, d_M, "fp64", ref)
    B.cos_sync_status()
    assert np.array_equal(out, ref.cpu().numpy())
    for c, n in enumerate(orders):
        terms = Ms[c] * gM[c]
        lhs = terms.sum() + float(np.dot(sigma, gs[c]))
        scale = np.abs(terms).sum() + float(np.abs(np.multiply(sigma, gs[c])).sum()) + 2 * n * abs(out[c])
        assert abs(lhs - 2 * n * out[c]) <= 1e-9 * scale, (c, n, lhs, 2 * n * out[c])
        assert abs(outT[c] - out[c]) <= 1e-9 * scale / (2 * n)
        assert np.max(np.abs(gMT[c] - np.swapaxes(gM[c], 1, 2))) <= 1e-9 * np.max(np.abs(gM[c]))
        assert np.max(np.abs(gsT[c] - gs[c])) <= 1e-9 * np.max(np.abs(gs[c]))


def test_grad_order10_sampled_entries():
    """The adjoint workload at the benchmark's size (SU(4), mu broken, n = 10, 5 x 10^4
    configurations, one gradient call): sampled entries of dc/dM against central
    differences of the oracle."""
    w = I.WORKLOADS["su4_adjoint_n10"]
    nc = w.n_cfg
    cfgs = I.workload_configs(w)
    tabs = B.tables_for(w.model)
    d = B.configs_to_device(cfgs)
    n_mat = 4
    gmoff = torch.arange(nc, dtype=torch.int64, device="cuda") * n_mat * 100
    gM = torch.empty(nc * n_mat * 100, dtype=torch.float64, device="cuda")
    out = torch.empty(nc, dtype=torch.float64, device="cuda")
    gmu = torch.empty(nc, 4, dtype=torch.float64, device="cuda")
    B.cos_connected_sum_grad(tabs, 10, *d, torch.ones(nc, dtype=torch.float64, device="cuda"), out, gM, gmoff,
                             gmu=gmu)
    B.cos_sync_status()
    g = gM.cpu().numpy().reshape(nc, n_mat, 10, 10)
    assert np.all(np.isfinite(gmu.cpu().numpy()))
    otabs = P.model_tables(w.model)
    rng = np.random.default_rng(0)
    for c in (0, nc // 2, nc - 1):
        M = P.gather_one(otabs, cfgs.site[cfgs.offset[c]:cfgs.offset[c] + 10],
                         cfgs.tau[cfgs.offset[c]:cfgs.offset[c] + 10], w.model.L, w.model.beta)
        mass = O.dp(M, None, absmode=True)
        assert abs(out.cpu().numpy()[c] - O.dp(M, None, prec="ld")) <= 1e-12 * mass
        for _ in range(4):
            idx = (int(rng.integers(4)), int(rng.integers(10)), int(rng.integers(10)))
            h = 0.05
            Mp = M.copy(); Mp[idx] += h
            Mm = M.copy(); Mm[idx] -= h
            ref = (O.dp(Mp, None, prec="ld") - O.dp(Mm, None, prec="ld")) / (2 * h)
            assert abs(g[c][idx] - ref) <= 1e-9 * (abs(ref) + np.max(np.abs(g[c]))), (c, idx, g[c][idx], ref)
    tabs.close()


def oracle_c(model, mu, alpha, cfgs, c):
    m = I.Model(model.L, model.t, model.beta, model.U, tuple(mu), tuple(alpha), model.n_tau)
    tabs = P.model_tables(m)
    n = int(cfgs.order[c])
    o = int(cfgs.offset[c])
    M = P.gather_one(tabs, cfgs.site[o:o + n], cfgs.tau[o:o + n], m.L, m.beta)
    sig = list(m.sigma)
    return O.dp(M, sig if any(sig) else None, prec="ld")


@pytest.mark.parametrize("sym", [False, True])
def test_grad_mu_alpha_chain_rule_vs_finite_differences(sym):
    nf = 3
    mu = [0.1] * nf if sym else [-0.2, 0.05, 0.3]
    alpha = [0.0] * nf if sym else [0.1, 0.0, -0.15]
    model = I.Model(8, 1.0, 3.0, 1.5, tuple(mu), tuple(alpha), 257)
    cfgs = I.make_configs(model, 5, 5, 6, seed=9)
    d = B.configs_to_device(cfgs)
    mu_t = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
    al_t = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    c = AG.connected_sum_model(mu_t, al_t, model, d, 5)
    c[2].backward()
    h = 1e-6
    for which, base, grad in (("mu", mu, mu_t.grad.numpy()), ("alpha", alpha, al_t.grad.numpy())):
        for l in range(nf):
            if sym:
                # symmetric tables: every flavor moves together, the gradient is split evenly
                p = [x + h for x in base]
                m = [x - h for x in base]
                fdv = (oracle_c(model, *((p, alpha) if which == "mu" else (mu, p)), cfgs, 2)
                       - oracle_c(model, *((m, alpha) if which == "mu" else (mu, m)), cfgs, 2)) / (2 * h) / nf
            else:
                p = list(base); p[l] += h
                m = list(base); m[l] -= h
                fdv = (oracle_c(model, *((p, alpha) if which == "mu" else (mu, p)), cfgs, 2)
                       - oracle_c(model, *((m, alpha) if which == "mu" else (mu, m)), cfgs, 2)) / (2 * h)
            assert grad[l] == pytest.approx(fdv, rel=2e-5, abs=1e-7 * max(1.0, abs(fdv))), (which, l, grad[l], fdv)


# ------------------------------------------------------------------ checkpointed layers

@pytest.mark.parametrize("n,n_mat,wt,shifts", [(6, 2, 1, True), (6, 3, 1, False), (5, 1, 4, True)])
def test_grad_checkpointed_matches_kept_layers_and_exact_differences(monkeypatch, n, n_mat, wt, shifts):
    """With the least-storage checkpoint plan forced (segments re-run from their checkpoints)
    the gradient is bitwise the one with every layer kept, and matches exact central
    differences of the __float128 oracle."""
    mask, store, rec = B.cos_grad_checkpoint_plan(n, 0)
    assert mask != 0 and rec > 0 and store < B.cos_structure(n).slots   # the forced plan does re-run layers
    Ms = list(I.random_matrices(900 + 10 * n + n_mat, 11, n_mat, n, 0.9))
    sigma = list(np.linspace(-0.12, 0.17, n_mat)) if shifts else None
    gout = np.linspace(0.5, 1.5, 11)
    monkeypatch.setenv("COS_GRAD_CHECKPOINT", "0")
    out0, gM0, gs0 = gpu_grad(Ms, n_mat, wt, sigma, gout)
    monkeypatch.setenv("COS_GRAD_CHECKPOINT", "1")
    out1, gM1, gs1 = gpu_grad(Ms, n_mat, wt, sigma, gout)
    assert np.array_equal(out0, out1)
    assert all(np.array_equal(a, b) for a, b in zip(gM0, gM1))
    assert np.array_equal(gs0, gs1)
    for c in (0, 10):
        assert close(gM1[c], gout[c] * exact_dM(Ms[c], sigma, wt)), c
        assert close(gs1[c], gout[c] * exact_dsigma(Ms[c], sigma, wt), rel=1e-7), c


def test_grad_checkpointed_orders_11_12_bitwise(monkeypatch):
    """Orders 11 and 12 with the least-storage plans forced: bitwise the gradient with every
    layer kept (uneven orders in one launch, each order with its own plan)."""
    orders = [12, 11, 12]
    n_mat = 2
    sigma = [0.05, -0.08]
    Ms = [I.random_matrices(1300 + c, 1, n_mat, n, 0.9)[0] for c, n in enumerate(orders)]
    gout = np.array([1.0, -0.5, 2.0])
    monkeypatch.setenv("COS_GRAD_CHECKPOINT", "0")
    out0, gM0, gs0 = gpu_grad(Ms, n_mat, 1, sigma, gout)
    monkeypatch.setenv("COS_GRAD_CHECKPOINT", "1")
    out1, gM1, gs1 = gpu_grad(Ms, n_mat, 1, sigma, gout)
    assert np.array_equal(out0, out1)
    assert all(np.array_equal(a, b) for a, b in zip(gM0, gM1))
    assert np.array_equal(gs0, gs1)


def test_det_grad_checkpointed_bitwise(monkeypatch):
    """Determinant weights (the Alg. 1 reverse sweep) with the least-storage plan forced."""
    n = 8
    Ms = I.random_matrices(77, 9, 2, n, 0.9)
    d_order, d_moff, d_M, order, moff = pack(list(Ms), 2)
    al = [0.1, -0.04]
    res = []
    for mode in ("0", "1"):
        monkeypatch.setenv("COS_GRAD_CHECKPOINT", mode)
        out = torch.empty(9, dtype=torch.float64, device="cuda")
        gM = torch.empty_like(d_M)
        ga = torch.empty(9, 2, dtype=torch.float64, device="cuda")
        B.cos_connected_det_matrices_grad(n, d_order, d_moff, al, d_M, torch.ones(9, dtype=torch.float64,
                                                                                 device="cuda"), out, gM, ga)
        B.cos_sync_status()
        res.append((out.cpu().numpy(), gM.cpu().numpy(), ga.cpu().numpy()))
    assert all(np.array_equal(a, b) for a, b in zip(res[0], res[1]))
