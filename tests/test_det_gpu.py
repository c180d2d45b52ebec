"""GPU parity of the SU(2) determinant-weight path (the DP without cycle factors, Alg. 1)
against the oracle.

The gradient: with determinant weights c is linear in every single matrix entry (an entry
occurs at most once in a determinant term, and in one factor of each product of the subset
subtraction; pinned by vanishing second differences in test_oracle_det_pins), so a central
difference of the
__float128 oracle is exact up to rounding.  dc/dalpha_b (a whole diagonal shifted) is checked
by an exact polynomial fit in alpha and by the identity dc/dalpha_b = -sum_j dc/dM_b[j][j].

The oracle value is `oracle.det_clow` (Alg. 1 as stated, point-resolved, long double),
itself pinned against LU determinants with the subset subtraction, brute force and the CoS
relation in test_oracle_det_pins.  Tolerances are the square-lattice ones of
test_parity_gpu, stated against the DP's mass (the same DP on |M| with |alpha| added to the
diagonal and every sign +): FP64 64 n 2^-53 mass, mixed (2n + log2(32 n)) 2^-24 mass,
double-float (16 n^2 + 64 n) 2^-48 mass.  Orders the oracle cannot reach in seconds (11, 12
on the square lattice, 9 on the bipartite one) use the CoS relation on the GPU: with two
flavors, loop weight 1 and no shifts the CoS sum of the same matrices is 2^n times this one.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from oracle import honeycomb as HC
from oracle import propagators as P
from paper_2507_12349_b300 import autograd as AG
from paper_2507_12349_b300 import binding as B
from paper_2507_12349_b300 import inputs as I

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24


def bound(prec, n, mass):
    if prec == "fp64":
        return 64 * n * EPS64 * mass
    if prec == "mixed":
        return (2 * n + math.log2(32 * n)) * EPS32 * mass
    return (16 * n * n + 64 * n) * 2.0 ** -48 * mass


def run_square(Ms, alpha=None, precision="fp64", abs_mass=True):
    order = np.array([m.shape[-1] for m in Ms], dtype=np.int32)
    moff = B.matrix_offsets(order, 2)
    flat = np.concatenate([np.asarray(m, dtype=np.float64).ravel() for m in Ms])
    d_order = torch.tensor(order, device="cuda")
    d_moff = torch.tensor(moff, device="cuda")
    d_M = torch.tensor(flat, device="cuda")
    out = torch.full((len(Ms),), float("nan"), dtype=torch.float64, device="cuda")
    mass = torch.full_like(out, float("nan")) if abs_mass else None
    B.cos_connected_det_matrices(int(order.max()), d_order, d_moff, alpha, d_M, precision, out, mass)
    B.cos_sync_status()
    return out.cpu().numpy(), (mass.cpu().numpy() if abs_mass else None)


def run_cos_square(Ms):
    """The CoS sum of the same two matrices (two flavors, loop weight 1, no shifts)."""
    order = np.array([m.shape[-1] for m in Ms], dtype=np.int32)
    d_order = torch.tensor(order, device="cuda")
    d_moff = torch.tensor(B.matrix_offsets(order, 2), device="cuda")
    d_M = torch.tensor(np.concatenate([m.ravel() for m in Ms]), device="cuda")
    out = torch.full((len(Ms),), float("nan"), dtype=torch.float64, device="cuda")
    mass = torch.full_like(out, float("nan"))
    B.cos_connected_sum_matrices(int(order.max()), d_order, d_moff, 2, 1, None, d_M, "fp64", out, mass)
    B.cos_sync_status()
    return out.cpu().numpy(), mass.cpu().numpy()


def run_bip(M4s, alpha2=None, precision="fp64", abs_mass=True, cos=False):
    order = np.array([m.shape[1] for m in M4s], dtype=np.int32)
    moff = B.bipartite_matrix_offsets(order, 2)
    d_order = torch.tensor(order, device="cuda")
    d_moff = torch.tensor(moff, device="cuda")
    d_M = torch.tensor(np.concatenate([m.ravel() for m in M4s]), device="cuda")
    out = torch.full((len(M4s),), float("nan"), dtype=torch.float64, device="cuda")
    mass = torch.full_like(out, float("nan")) if abs_mass else None
    if cos:
        B.cos_connected_sum_bipartite_matrices(int(order.max()), d_order, d_moff, 2, 1, None, d_M, precision, out,
                                               mass)
    else:
        B.cos_connected_det_bipartite_matrices(int(order.max()), d_order, d_moff, alpha2, d_M, precision, out, mass)
    B.cos_sync_status()
    return out.cpu().numpy(), (mass.cpu().numpy() if abs_mass else None)


def rand_sq(seed, ncfg, n, scale=0.9):
    return list(I.random_matrices(seed, ncfg, 2, n, scale))


def rand_m4(seed, ncfg, n, scale=0.9):
    M = I.random_matrices(seed, ncfg, 2, 2 * n, scale)
    return [np.ascontiguousarray(m.reshape(2, n, 2, n, 2)) for m in M]


SQUARE = [  # n, configurations, shifts
    (1, 5, True), (2, 9, False), (3, 17, True), (4, 33, False), (5, 12, True), (6, 7, True), (7, 20, False),
    (8, 6, True), (9, 3, False), (10, 3, True),
]


@pytest.mark.parametrize("n,ncfg,shifts", SQUARE)
@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
def test_square_matches_oracle(n, ncfg, shifts, prec):
    if prec != "fp64" and n > 8:
        pytest.skip("reduced precisions are checked up to n = 8 here and at n = 10 on the workload")
    Ms = rand_sq(2000 + 10 * n, ncfg, n)
    al = [0.13, -0.08] if shifts else None
    got, mass = run_square(Ms, al, prec)
    for c in sorted({0, ncfg // 2, ncfg - 1}):
        ref = O.det_clow(Ms[c], al, prec="ld")
        rmass = O.det_clow(Ms[c], al, absmode=True)
        assert abs(got[c] - ref) <= bound(prec, n, rmass), (c, got[c], ref, rmass)
        assert mass[c] == pytest.approx(rmass, rel=1e-12 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
def test_square_uneven_orders_and_cos_relation(prec):
    """Orders 1..12 in one launch; up to 8 against the oracle, every order against the FP64
    CoS kernel on the same matrices (c_CoS = 2^n c)."""
    orders = [12, 3, 11, 1, 7, 10, 2, 12, 5, 9, 4, 6, 8, 11]
    Ms = [rand_sq(3000 + c, 1, n)[0] for c, n in enumerate(orders)]
    got, mass = run_square(Ms, None, prec)
    cos, cmass = run_cos_square(Ms)
    for c, n in enumerate(orders):
        if n <= 8:
            ref = O.det_clow(Ms[c], prec="ld")
            rmass = O.det_clow(Ms[c], absmode=True)
            assert abs(got[c] - ref) <= bound(prec, n, rmass), (c, n, got[c], ref)
        # the two GPU paths agree through the CoS relation at every order
        tol = bound(prec, n, mass[c]) + bound("fp64", n, cmass[c]) / 2.0 ** n
        assert abs(got[c] - cos[c] / 2.0 ** n) <= tol, (c, n, got[c], cos[c] / 2.0 ** n)


def test_square_deterministic():
    Ms = rand_sq(44, 50, 7)
    a, _ = run_square(Ms, [0.1, 0.2], abs_mass=False)
    b, _ = run_square(Ms, [0.1, 0.2], abs_mass=False)
    assert np.array_equal(a, b)


BIP = [  # n, configurations, shifts
    (1, 5, True), (2, 9, False), (3, 17, True), (4, 12, False), (5, 7, True), (6, 5, False), (7, 3, True),
    (8, 2, True),
]


def bip_bound(prec, n, mass):
    """Bipartite rows hold up to 2n - 1 states: the mixed bound takes log2 of the doubled fan-in."""
    if prec == "mixed":
        return (2 * n + math.log2(64 * n)) * EPS32 * mass
    return bound(prec, n, mass)


@pytest.mark.parametrize("n,ncfg,shifts", BIP)
@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
def test_bipartite_matches_oracle(n, ncfg, shifts, prec):
    M4s = rand_m4(5000 + 10 * n, ncfg, n)
    al = [[0.11, -0.05], [-0.07, 0.09]] if shifts else None
    got, mass = run_bip(M4s, al, prec)
    for c in sorted({0, ncfg // 2, ncfg - 1}):
        ref = O.det_clow(M4s[c], al, prec="ld")
        rmass = O.det_clow(M4s[c], al, absmode=True)
        assert abs(got[c] - ref) <= bip_bound(prec, n, rmass), (c, got[c], ref, rmass)
        assert mass[c] == pytest.approx(rmass, rel={"fp64": 1e-12, "df64": 1e-9, "mixed": 1e-5}[prec])


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_bipartite_uneven_and_order9_cos_relation(prec):
    orders = [9, 2, 6, 1, 9, 4, 8, 3, 5, 7]
    M4s = [rand_m4(6000 + c, 1, n)[0] for c, n in enumerate(orders)]
    got, mass = run_bip(M4s, None, prec)
    cos, cmass = run_bip(M4s, cos=True)
    for c, n in enumerate(orders):
        if n <= 6:
            ref = O.det_clow(M4s[c], prec="ld")
            rmass = O.det_clow(M4s[c], absmode=True)
            assert abs(got[c] - ref) <= bound(prec, n, rmass), (c, n, got[c], ref)
        tol = bound(prec, n, mass[c]) + bound("fp64", n, cmass[c]) / 2.0 ** n
        assert abs(got[c] - cos[c] / 2.0 ** n) <= tol, (c, n, got[c], cos[c] / 2.0 ** n)


def test_bipartite_deterministic():
    M4s = rand_m4(55, 40, 5)
    a, _ = run_bip(M4s, [[0.1, 0.0], [0.0, -0.1]], abs_mass=False)
    b, _ = run_bip(M4s, [[0.1, 0.0], [0.0, -0.1]], abs_mass=False)
    assert np.array_equal(a, b)


def test_bipartite_rejects_unknown_precision():
    M4s = rand_m4(1, 1, 2)
    with pytest.raises(KeyError):
        run_bip(M4s, None, "fp16")


@pytest.mark.parametrize("prec,sample", [("fp64", 6), ("df64", 4), ("mixed", 4)])
def test_workload_su2_zeeman_order10_sampled(prec, sample):
    """The order-10 SU(2) workload at full size (20 000 configurations, the launch the
    benchmark times): gather with the two-flavor tables, DP on the GPU, sampled
    configurations against the oracle's gather and Alg. 1."""
    w = I.WORKLOADS["su2_zeeman_det_n10"]
    cfgs = I.workload_configs(w)
    n_cfg = cfgs.n_cfg
    tabs = B.tables_for(w.model)
    d = B.configs_to_device(cfgs)
    moff = B.matrix_offsets(cfgs.order, 2)
    d_moff = torch.tensor(moff, device="cuda")
    M = torch.empty(int(moff[-1]) + 2 * 100, dtype=torch.float64, device="cuda")
    B.cos_gather(tabs, *d, d_moff, M)
    out = torch.full((n_cfg,), float("nan"), dtype=torch.float64, device="cuda")
    mass = torch.full_like(out, float("nan"))
    B.cos_connected_det_matrices(10, d[0], d_moff, None, M, prec, out, mass)
    B.cos_sync_status()
    got, gmass = out.cpu().numpy(), mass.cpu().numpy()
    assert np.all(np.isfinite(got))
    otabs = P.model_tables(w.model)
    idx = sorted(set(np.linspace(0, n_cfg - 1, sample).astype(int)))
    for c, Mc in zip(idx, P.gather(otabs, cfgs, w.model.L, w.model.beta, idx)):
        ref = O.det_clow(Mc, prec="ld")
        rmass = O.det_clow(Mc, absmode=True)
        assert abs(got[c] - ref) <= bound(prec, 10, rmass), (c, got[c], ref, rmass)
        if prec == "fp64":
            assert gmass[c] == pytest.approx(rmass, rel=1e-10)
    tabs.close()


def test_honeycomb_det_sampled():
    """Honeycomb SU(2) tables (the order-8 workload's model), gathered on the GPU, with the
    staggered shifts as diagonal shifts of the determinant weights."""
    w = I.WORKLOADS["hc_su2_af_n8"]
    cfgs = I.workload_configs(w, 64)
    tabs = B.honeycomb_tables_for(w.model)
    d = B.configs_to_device(cfgs)
    moff = B.bipartite_matrix_offsets(cfgs.order, 2)
    d_moff = torch.tensor(moff, device="cuda")
    M4 = torch.empty(int(moff[-1]) + 2 * 16 * 16, dtype=torch.float64, device="cuda")
    B.cos_gather_bipartite(tabs, *d, d_moff, M4)
    al = [list(r) for r in w.model.sigma2]
    out = torch.full((64,), float("nan"), dtype=torch.float64, device="cuda")
    B.cos_connected_det_bipartite_matrices(8, d[0], d_moff, al, M4, "fp64", out)
    B.cos_sync_status()
    got = out.cpu().numpy()
    otabs = HC.hc_model_tables(w.model)
    for c in (0, 63):
        o = int(cfgs.offset[c])
        M4c = HC.hc_gather_one(otabs, cfgs.site[o:o + 8], cfgs.tau[o:o + 8], w.model.L, w.model.beta)
        ref = O.det_clow(M4c, al, prec="ld")
        rmass = O.det_clow(M4c, al, absmode=True)
        assert abs(got[c] - ref) <= bound("fp64", 8, rmass), (c, got[c], ref, rmass)
    tabs.close()


# ------------------------------------------------------------------ gradient

def run_grad(Ms, alpha, gout):
    order = np.array([m.shape[-1] for m in Ms], dtype=np.int32)
    moff = B.matrix_offsets(order, 2)
    d_order = torch.tensor(order, device="cuda")
    d_moff = torch.tensor(moff, device="cuda")
    d_M = torch.tensor(np.concatenate([m.ravel() for m in Ms]), device="cuda")
    nc = len(Ms)
    out = torch.full((nc,), float("nan"), dtype=torch.float64, device="cuda")
    gM = torch.full_like(d_M, float("nan"))
    ga = torch.full((nc, 2), float("nan"), dtype=torch.float64, device="cuda")
    B.cos_connected_det_matrices_grad(int(order.max()), d_order, d_moff, alpha, d_M,
                                      torch.tensor(gout, dtype=torch.float64, device="cuda"), out, gM, ga)
    B.cos_sync_status()
    g = gM.cpu().numpy()
    return out.cpu().numpy(), [g[moff[c]:moff[c] + Ms[c].size].reshape(Ms[c].shape) for c in range(nc)], ga.cpu().numpy()


def exact_det_dM(G, alpha, h=0.5):
    g = np.zeros_like(G)
    for idx in np.ndindex(*G.shape):
        Gp = G.copy(); Gp[idx] += h
        Gm = G.copy(); Gm[idx] -= h
        g[idx] = (O.det_clow(Gp, alpha, prec="q") - O.det_clow(Gm, alpha, prec="q")) / (2 * h)
    return g


def exact_det_dalpha(G, alpha):
    n = G.shape[-1]
    a0 = np.zeros(2) if alpha is None else np.array(alpha, dtype=np.float64)
    out = []
    for b in range(2):
        hs = [0.05 * k for k in range(-n - 1, n + 2)]
        vals = []
        for h in hs:
            a2 = a0.copy(); a2[b] += h
            vals.append(O.det_clow(G, a2, prec="q"))
        out.append(np.polyfit(hs, vals, n + 1)[-2])
    return np.array(out)


def close_to(a, b, rel=1e-9):
    scale = max(np.max(np.abs(b)), 1e-300)
    return np.all(np.abs(a - b) <= rel * (np.abs(b) + scale))


@pytest.mark.parametrize("n,ncfg,shifts", [(1, 3, True), (2, 5, False), (3, 7, True), (4, 9, True), (5, 4, False)])
def test_det_grad_vs_exact_differences(n, ncfg, shifts):
    Ms = rand_sq(7000 + n, ncfg, n)
    al = [0.11, -0.06] if shifts else None
    gout = np.linspace(0.5, 1.5, ncfg)
    out, gM, ga = run_grad(Ms, al, gout)
    for c in sorted({0, ncfg // 2, ncfg - 1}):
        ref = O.det_clow(Ms[c], al, prec="ld")
        assert abs(out[c] - ref) <= bound("fp64", n, O.det_clow(Ms[c], al, absmode=True))
        dM = gout[c] * exact_det_dM(Ms[c], al)
        assert close_to(gM[c], dM), c
        assert close_to(ga[c], gout[c] * exact_det_dalpha(Ms[c], al), rel=1e-7), c
        assert close_to(ga[c], -np.array([np.trace(dM[0]), np.trace(dM[1])])), c


def test_det_grad_orders_11_12_euler():
    """Orders 11 and 12: c(t M, t alpha) = t^(2n) c gives sum M dc/dM + sum alpha dc/dalpha = 2n c;
    the forward value equals the determinant sweep's bit for bit."""
    orders = [12, 11, 12, 11, 7]
    al = [0.09, -0.04]
    Ms = [rand_sq(7100 + c, 1, n)[0] for c, n in enumerate(orders)]
    out, gM, ga = run_grad(Ms, al, np.ones(len(Ms)))
    ref, _ = run_square(Ms, al, abs_mass=False)
    assert np.array_equal(out, ref)
    for c, n in enumerate(orders):
        terms = Ms[c] * gM[c]
        lhs = terms.sum() + float(np.dot(al, ga[c]))
        scale = np.abs(terms).sum() + float(np.abs(np.multiply(al, ga[c])).sum()) + 2 * n * abs(out[c])
        assert abs(lhs - 2 * n * out[c]) <= 1e-9 * scale, (c, n, lhs, 2 * n * out[c])


# ------------------------------------------------------------------ every vertex subset

def run_det_subsets(Ms, alpha, n_max=None, want_a=True, all_roots=True):
    order = np.array([m.shape[-1] for m in Ms], dtype=np.int32)
    moff = B.matrix_offsets(order, 2)
    n_max = int(order.max()) if n_max is None else n_max
    d_order = torch.tensor(order, device="cuda")
    d_moff = torch.tensor(moff, device="cuda")
    d_M = torch.tensor(np.concatenate([m.ravel() for m in Ms]), device="cuda")
    per = 1 << n_max
    c = torch.full((len(Ms) * per,), 12345.0, dtype=torch.float64, device="cuda")
    a = torch.full_like(c, 12345.0) if want_a else None
    B.cos_connected_det_subsets(n_max, d_order, d_moff, alpha, d_M, c, a, all_roots)
    B.cos_sync_status()
    return c.cpu().numpy().reshape(len(Ms), per), (a.cpu().numpy().reshape(len(Ms), per) if want_a else None)


@pytest.mark.parametrize("orders,shifts", [([5, 5, 5], True), ([6, 3, 1, 4], False), ([7, 2], True)])
def test_det_subsets_every_subset(orders, shifts):
    """c(S) of every subset against Alg. 1 of the oracle on the principal sub-matrices, a(S)
    against LU determinants (a route that never forms c)."""
    al = [0.12, -0.07] if shifts else None
    Ms = [rand_sq(8000 + 10 * c + n, 1, n)[0] for c, n in enumerate(orders)]
    n_max = max(orders)
    c_got, a_got = run_det_subsets(Ms, al, n_max)
    for ci, M in enumerate(Ms):
        n = M.shape[-1]
        for S in range(1, 1 << n):
            idx = [i for i in range(n) if S >> i & 1]
            sub = np.ascontiguousarray(M[:, idx][:, :, idx])
            ref = O.det_clow(sub, al, prec="q")
            rmass = O.det_clow(sub, al, absmode=True)
            assert abs(c_got[ci, S] - ref) <= bound("fp64", len(idx), rmass), (ci, S, c_got[ci, S], ref)
            A = [sub[b] - (0.0 if al is None else al[b]) * np.eye(len(idx)) for b in range(2)]
            aref = np.linalg.det(A[0]) * np.linalg.det(A[1])
            assert abs(a_got[ci, S] - aref) <= 1e-11 * (abs(aref) + rmass), (ci, S, a_got[ci, S], aref)
        assert a_got[ci, 0] == 1.0 and c_got[ci, 0] == 0.0
        assert np.all(c_got[ci, 1 << n:] == 0.0) and np.all(a_got[ci, 1 << n:] == 0.0)


def test_det_subsets_root0_only_and_full_value():
    """all_roots = 0: the subsets containing vertex 0, from one sweep; c(V) equals the plain
    determinant sweep bit for bit."""
    Ms = rand_sq(8100, 6, 6)
    al = [0.05, 0.02]
    c_got, _ = run_det_subsets(Ms, al, want_a=False, all_roots=False)
    plain, _ = run_square(Ms, al, abs_mass=False)
    for ci, M in enumerate(Ms):
        assert c_got[ci, 63] == plain[ci]
        for S in (1, 3, 5, 33, 47):
            idx = [i for i in range(6) if S >> i & 1]
            sub = np.ascontiguousarray(M[:, idx][:, :, idx])
            ref = O.det_clow(sub, al, prec="q")
            assert abs(c_got[ci, S] - ref) <= bound("fp64", len(idx), O.det_clow(sub, al, absmode=True))


def test_det_autograd_function():
    """torch.autograd through connected_det equals the reverse sweep's gradient, weighted."""
    Ms = rand_sq(8300, 5, 5)
    order = np.array([5] * 5, dtype=np.int32)
    moff = B.matrix_offsets(order, 2)
    M = torch.tensor(np.concatenate([m.ravel() for m in Ms]), device="cuda", requires_grad=True)
    al = torch.tensor([0.1, -0.05], dtype=torch.float64, requires_grad=True)
    w = torch.linspace(0.5, 1.5, 5, dtype=torch.float64, device="cuda")
    c = AG.connected_det(M, al, torch.tensor(order, device="cuda"), torch.tensor(moff, device="cuda"), 5)
    (c * w).sum().backward()
    out, gM, ga = run_grad(Ms, [0.1, -0.05], w.cpu().numpy())
    assert np.array_equal(c.detach().cpu().numpy(), out)
    assert np.allclose(M.grad.cpu().numpy(), np.concatenate([g.ravel() for g in gM]), rtol=0, atol=0)
    assert np.allclose(al.grad.numpy(), ga.sum(0), rtol=1e-14, atol=0)


@pytest.mark.parametrize("sym", [False, True])
def test_det_batch_from_coordinates(sym):
    """Gather + determinant sweep in one call, against the oracle's gather and Alg. 1; with
    equal chemical potentials the collapsed tables serve both spin blocks."""
    w = I.WORKLOADS["su2_zeeman_det_n10"]
    m = w.model
    model = I.Model(m.L, m.t, m.beta, m.U, (0.1, 0.1) if sym else m.mu, (0.0, 0.0), m.n_tau)
    cfgs = I.make_configs(model, 3, 8, 300, 17)
    tabs = B.tables_for(model)
    assert tabs.info().n_mat == (1 if sym else 2)
    d = B.configs_to_device(cfgs)
    al = [0.07, -0.03]
    out = torch.full((300,), float("nan"), dtype=torch.float64, device="cuda")
    mass = torch.full_like(out, float("nan"))
    B.cos_connected_det_batch(tabs, 8, *d, al, "fp64", out, mass)
    B.cos_sync_status()
    got, gmass = out.cpu().numpy(), mass.cpu().numpy()
    otabs = P.model_tables(model)
    if sym:
        otabs = np.concatenate([otabs[:1], otabs[:1]])
    for c, Mc in zip((0, 150, 299), P.gather(otabs, cfgs, model.L, model.beta, (0, 150, 299))):
        n = int(cfgs.order[c])
        ref = O.det_clow(Mc, al, prec="ld")
        rmass = O.det_clow(Mc, al, absmode=True)
        assert abs(got[c] - ref) <= bound("fp64", n, rmass) + 1e-13 * rmass, (c, got[c], ref)
        assert gmass[c] == pytest.approx(rmass, rel=1e-10)
    tabs.close()


@pytest.mark.parametrize("sym", [False, True])
def test_det_grad_from_coordinates(sym):
    """dLoss/dM, dLoss/dalpha and dLoss/dmu from vertex coordinates.  dM and dalpha: the same
    reverse sweep as the matrices entry on the blocks cos_gather writes (bitwise).  dmu: a
    central difference of the oracle pipeline (tables, gather and Alg. 1 rebuilt at mu +- h);
    collapsed tables (equal chemical potentials) move both spins together and split the
    derivative evenly."""
    base = I.WORKLOADS["su2_zeeman_det_n10"].model
    mu = [0.1, 0.1] if sym else [-0.15, 0.2]
    model = I.Model(base.L, base.t, base.beta, base.U, tuple(mu), (0.0, 0.0), base.n_tau)
    nc = 40
    cfgs = I.make_configs(model, 3, 6, nc, 23)
    tabs = B.tables_for(model)
    n_mat = tabs.info().n_mat
    assert n_mat == (1 if sym else 2)
    d = B.configs_to_device(cfgs)
    al = [0.06, -0.04]
    order = cfgs.order.astype(np.int32)
    gmoff = B.matrix_offsets(order, 2)
    gout = np.linspace(0.5, 1.5, nc)
    out = torch.full((nc,), float("nan"), dtype=torch.float64, device="cuda")
    gM = torch.full((int(2 * (order.astype(np.int64) ** 2).sum()),), float("nan"), dtype=torch.float64,
                    device="cuda")
    gmu = torch.full((nc, 2), float("nan"), dtype=torch.float64, device="cuda")
    ga = torch.full_like(gmu, float("nan"))
    B.cos_connected_det_grad(tabs, 6, *d, al, torch.tensor(gout, device="cuda"), out, gM,
                             torch.tensor(gmoff, device="cuda"), gmu, ga)
    B.cos_sync_status()
    out, gM, gmu, ga = (x.cpu().numpy() for x in (out, gM, gmu, ga))

    moff = B.matrix_offsets(order, n_mat)
    Mg = torch.empty(int(n_mat * (order.astype(np.int64) ** 2).sum()), dtype=torch.float64, device="cuda")
    B.cos_gather(tabs, *d, torch.tensor(moff, device="cuda"), Mg)
    host = Mg.cpu().numpy()
    Ms = []
    for c in range(nc):
        n = int(order[c])
        blk = host[moff[c]:moff[c] + n_mat * n * n].reshape(n_mat, n, n)
        Ms.append(np.ascontiguousarray(np.concatenate([blk, blk]) if n_mat == 1 else blk))
    ref_out, ref_gM, ref_ga = run_grad(Ms, al, gout)
    assert np.array_equal(out, ref_out)
    assert np.array_equal(gM, np.concatenate([g.ravel() for g in ref_gM]))
    assert np.array_equal(ga, ref_ga)

    def oracle_c(mu2, c):
        m = I.Model(model.L, model.t, model.beta, model.U, tuple(mu2), (0.0, 0.0), model.n_tau)
        t = P.model_tables(m)
        if t.shape[0] == 1:
            t = np.concatenate([t, t])
        o, n = int(cfgs.offset[c]), int(cfgs.order[c])
        return O.det_clow(P.gather_one(t, cfgs.site[o:o + n], cfgs.tau[o:o + n], m.L, m.beta), al, prec="ld")

    h = 1e-6
    for c in (0, nc // 2, nc - 1):
        for b in range(2):
            if sym:
                fd = (oracle_c([x + h for x in mu], c) - oracle_c([x - h for x in mu], c)) / (2 * h) / 2
            else:
                p = list(mu); p[b] += h
                q = list(mu); q[b] -= h
                fd = (oracle_c(p, c) - oracle_c(q, c)) / (2 * h)
            want = gout[c] * fd
            assert gmu[c, b] == pytest.approx(want, rel=2e-5, abs=1e-7 * max(1.0, abs(want))), (c, b, gmu[c, b], want)
    tabs.close()


def test_det_model_autograd():
    """connected_det_model: the forward equals cos_connected_det_batch, and mu.grad / alpha.grad
    are the per-configuration gradients of cos_connected_det_grad summed with the weights."""
    base = I.WORKLOADS["su2_zeeman_det_n10"].model
    mu = [-0.1, 0.25]
    model = I.Model(base.L, base.t, base.beta, base.U, tuple(mu), (0.0, 0.0), base.n_tau)
    cfgs = I.make_configs(model, 4, 7, 64, 5)
    d = B.configs_to_device(cfgs)
    mu_t = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
    al_t = torch.tensor([0.03, 0.08], dtype=torch.float64, requires_grad=True)
    c = AG.connected_det_model(mu_t, al_t, model, d, 7)
    w = torch.linspace(-1.0, 2.0, 64, dtype=torch.float64, device="cuda")
    (c * w).sum().backward()
    tabs = B.tables_for(model)
    ref = torch.empty(64, dtype=torch.float64, device="cuda")
    B.cos_connected_det_batch(tabs, 7, *d, [0.03, 0.08], "fp64", ref)
    gmu = torch.empty(64, 2, dtype=torch.float64, device="cuda")
    gal = torch.empty_like(gmu)
    B.cos_connected_det_grad(tabs, 7, *d, [0.03, 0.08], w, gmu=gmu, galpha=gal)
    B.cos_sync_status()
    tabs.close()
    assert np.array_equal(c.detach().cpu().numpy(), ref.cpu().numpy())
    assert np.allclose(mu_t.grad.numpy(), gmu.sum(0).cpu().numpy(), rtol=1e-14, atol=0)
    assert np.allclose(al_t.grad.numpy(), gal.sum(0).cpu().numpy(), rtol=1e-14, atol=0)


@pytest.mark.parametrize("sym", [False, True])
def test_det_bipartite_batch_from_coordinates(sym):
    """Gather + bipartite determinant sweep in one call: bit for bit the two-step path
    (cos_gather_bipartite, then the matrices entry) and, on samples, the oracle's gather with
    Alg. 1; with equal spins the collapsed tables serve both blocks."""
    m = I.WORKLOADS["hc_su2_af_n8"].model
    model = I.HoneycombModel(m.L, m.t, m.beta, m.U, m.mu, m.alpha, (0.25, 0.25) if sym else m.delta, m.n_tau)
    nc = 300
    cfgs = I.make_configs(model, 3, 7, nc, 19)
    tabs = B.honeycomb_tables_for(model)
    n_mat = tabs.info().n_mat
    assert n_mat == (1 if sym else 2)
    d = B.configs_to_device(cfgs)
    al = [[0.05, -0.03], [0.02, 0.06]]
    out = torch.full((nc,), float("nan"), dtype=torch.float64, device="cuda")
    mass = torch.full_like(out, float("nan"))
    B.cos_connected_det_bipartite_batch(tabs, 7, *d, al, "fp64", out, mass)
    order = cfgs.order.astype(np.int32)
    moff = B.bipartite_matrix_offsets(order, n_mat)
    M4 = torch.empty(int(n_mat * 4 * (order.astype(np.int64) ** 2).sum()), dtype=torch.float64, device="cuda")
    B.cos_gather_bipartite(tabs, *d, torch.tensor(moff, device="cuda"), M4)
    host = M4.cpu().numpy()
    blocks = []
    for c in range(nc):
        w2 = 4 * int(order[c]) ** 2
        b = host[moff[c]:moff[c] + n_mat * w2]
        blocks.append(np.concatenate([b, b]) if n_mat == 1 else b)
    moff2 = torch.tensor(B.bipartite_matrix_offsets(order, 2), device="cuda")
    ref = torch.full_like(out, float("nan"))
    rmass = torch.full_like(out, float("nan"))
    B.cos_connected_det_bipartite_matrices(7, d[0], moff2, al, torch.tensor(np.concatenate(blocks), device="cuda"),
                                           "fp64", ref, rmass)
    B.cos_sync_status()
    tabs.close()
    got, gmass = out.cpu().numpy(), mass.cpu().numpy()
    assert np.array_equal(got, ref.cpu().numpy()) and np.array_equal(gmass, rmass.cpu().numpy())
    otabs = HC.hc_model_tables(model)
    for c in (0, nc // 2, nc - 1):
        o, n = int(cfgs.offset[c]), int(cfgs.order[c])
        G4 = HC.hc_gather_one(otabs, cfgs.site[o:o + n], cfgs.tau[o:o + n], model.L, model.beta)
        r = O.det_clow(G4, al, prec="ld")
        rm = O.det_clow(G4, al, absmode=True)
        assert abs(got[c] - r) <= bound("fp64", n, rm) + 1e-13 * rm, (c, got[c], r)


@pytest.mark.parametrize("sym", [False, True])
def test_det_bipartite_grad_from_coordinates(sym):
    """Bipartite determinant weights from vertex coordinates: dLoss/dM4 and dLoss/dalpha2 bit
    for bit the matrices entry's on the gathered blocks; dLoss/dmu against central differences
    of the oracle pipeline (honeycomb tables, gather, Alg. 1) rebuilt at mu +- h; collapsed
    tables move both spins together and split the derivative evenly."""
    m0 = I.WORKLOADS["hc_su2_af_n8"].model
    mu = [0.1, 0.1] if sym else [-0.15, 0.2]
    delta = (0.25, 0.25) if sym else m0.delta
    mk = lambda m: I.HoneycombModel(m0.L, m0.t, m0.beta, m0.U, tuple(m), (0.0, 0.0), delta, m0.n_tau)
    model = mk(mu)
    nc = 24
    cfgs = I.make_configs(model, 3, 5, nc, 37)
    tabs = B.honeycomb_tables_for(model)
    n_mat = tabs.info().n_mat
    assert n_mat == (1 if sym else 2)
    d = B.configs_to_device(cfgs)
    al = [[0.05, -0.03], [0.02, 0.06]]
    order = cfgs.order.astype(np.int32)
    moff2 = torch.tensor(B.bipartite_matrix_offsets(order, 2), device="cuda")
    total2 = int(8 * (order.astype(np.int64) ** 2).sum())
    gout = np.linspace(0.5, 1.5, nc)
    g = torch.tensor(gout, device="cuda")
    nan = float("nan")
    out = torch.full((nc,), nan, dtype=torch.float64, device="cuda")
    gM = torch.full((total2,), nan, dtype=torch.float64, device="cuda")
    gmu = torch.full((nc, 2), nan, dtype=torch.float64, device="cuda")
    ga = torch.full((nc, 2, 2), nan, dtype=torch.float64, device="cuda")
    B.cos_connected_det_bipartite_grad(tabs, 5, *d, al, g, out, gM, moff2, gmu, ga)
    moff = B.bipartite_matrix_offsets(order, n_mat)
    M4 = torch.empty(int(n_mat * 4 * (order.astype(np.int64) ** 2).sum()), dtype=torch.float64, device="cuda")
    B.cos_gather_bipartite(tabs, *d, torch.tensor(moff, device="cuda"), M4)
    host = M4.cpu().numpy()
    blocks = []
    for c in range(nc):
        b = host[moff[c]:moff[c] + n_mat * 4 * int(order[c]) ** 2]
        blocks.append(np.concatenate([b, b]) if n_mat == 1 else b)
    out2 = torch.full_like(out, nan)
    gM2 = torch.full_like(gM, nan)
    ga2 = torch.full_like(ga, nan)
    B.cos_connected_det_bipartite_matrices_grad(5, d[0], moff2, al, torch.tensor(np.concatenate(blocks), device="cuda"),
                                                g, out2, gM2, ga2)
    B.cos_sync_status()
    tabs.close()
    assert np.array_equal(out.cpu().numpy(), out2.cpu().numpy())
    assert np.array_equal(gM.cpu().numpy(), gM2.cpu().numpy())
    assert np.array_equal(ga.cpu().numpy(), ga2.cpu().numpy())
    gmu = gmu.cpu().numpy()
    picks = (0, nc // 2, nc - 1)

    def oracle_c(m2):
        m = mk(m2)
        t = HC.hc_model_tables(m)
        vals = []
        for c in picks:
            o, n = int(cfgs.offset[c]), int(cfgs.order[c])
            G4 = HC.hc_gather_one(t, cfgs.site[o:o + n], cfgs.tau[o:o + n], m.L, m.beta)
            vals.append(O.det_clow(G4, al, prec="ld"))
        return np.array(vals)

    h = 1e-6
    for b in range(2):
        if sym:
            fd = (oracle_c([x + h for x in mu]) - oracle_c([x - h for x in mu])) / (2 * h) / 2
        else:
            p = list(mu); p[b] += h
            q = list(mu); q[b] -= h
            fd = (oracle_c(p) - oracle_c(q)) / (2 * h)
        for k, c in enumerate(picks):
            want = gout[c] * fd[k]
            assert gmu[c, b] == pytest.approx(want, rel=2e-5, abs=1e-7 * max(1.0, abs(want))), (b, c, gmu[c, b], want)


def test_det_bipartite_model_autograd():
    """connected_det_bipartite_model: the forward equals cos_connected_det_bipartite_batch bit for
    bit; mu.grad and alpha2.grad are the per-configuration gradients summed with the weights."""
    m0 = I.WORKLOADS["hc_su2_af_n8"].model
    mu = [-0.1, 0.15]
    model = I.HoneycombModel(m0.L, m0.t, m0.beta, m0.U, tuple(mu), (0.0, 0.0), m0.delta, m0.n_tau)
    nc = 48
    cfgs = I.make_configs(model, 3, 6, nc, 43)
    d = B.configs_to_device(cfgs)
    al = [[0.04, -0.02], [0.03, 0.05]]
    mu_t = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
    al_t = torch.tensor(al, dtype=torch.float64, requires_grad=True)
    c = AG.connected_det_bipartite_model(mu_t, al_t, model, d, 6)
    w = torch.linspace(-1.0, 2.0, nc, dtype=torch.float64, device="cuda")
    (c * w).sum().backward()
    tabs = B.honeycomb_tables_for(model)
    ref = torch.empty(nc, dtype=torch.float64, device="cuda")
    B.cos_connected_det_bipartite_batch(tabs, 6, *d, al, "fp64", ref)
    gmu = torch.empty(nc, 2, dtype=torch.float64, device="cuda")
    gal = torch.empty(nc, 2, 2, dtype=torch.float64, device="cuda")
    B.cos_connected_det_bipartite_grad(tabs, 6, *d, al, w, gmu=gmu, galpha2=gal)
    B.cos_sync_status()
    tabs.close()
    assert np.array_equal(c.detach().cpu().numpy(), ref.cpu().numpy())
    assert np.allclose(mu_t.grad.numpy(), gmu.sum(0).cpu().numpy(), rtol=1e-14, atol=0)
    assert np.allclose(al_t.grad.numpy(), gal.sum(0).cpu().numpy(), rtol=1e-14, atol=0)
