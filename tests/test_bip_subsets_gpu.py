"""GPU parity of the bipartite all-subsets mode (cos_connected_sum_bipartite_subsets and
cos_connected_det_bipartite_subsets) against the oracle.

References (none of them runs the sublattice-resolved sweep):
  * c(S), cycle factors: the oracle's sum over the sublattice assignments of S of the closed
    form (determinants + the subset recursion of Methods A) on the sub-configuration S,
    __float128;
  * a(S), cycle factors: for every assignment s of all n vertices the closed form's full sums
    of every subset, summed over s and divided by 2^(n - |S|) (the assignments of the vertices
    outside S), so the GPU subset exponential is checked against a route that never forms c;
  * c(S), determinant weights: `oracle.det_clow` (Alg. 1 as stated, point-resolved) on the
    sub-configuration; a(S) = sum over the assignments of S of det(A_up) det(A_dn) by LU.
Tolerances, per subset, against the absolute mass (the same DP on |M4| with every sign +):
FP64 |c err| <= 64 |S| 2^-53 mass(S), |a err| <= 128 n 2^-53 amass(S), amass the subset
exponential of the masses (a bound on the sum of |terms| of a(S)).
"""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from oracle import honeycomb as HC
from paper_2507_12349_b300 import binding as B
from paper_2507_12349_b300 import inputs as I

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53


def members(S):
    return [i for i in range(S.bit_length()) if S >> i & 1]


def rand_m4(seed, ncfg, nf, n, scale=0.9):
    M = I.random_matrices(seed, ncfg, nf, 2 * n, scale)         # [cfg][nf][2n][2n], index i*2 + s
    return [np.ascontiguousarray(m.reshape(nf, n, 2, n, 2)) for m in M]


def sub4(M4, idx):
    return np.ascontiguousarray(M4[:, idx][:, :, :, idx])


def subset_exp(c, n):
    a = np.zeros(1 << n)
    a[0] = 1.0
    for S in range(1, 1 << n):
        low = S & -S
        rest = S ^ low
        R, acc = rest, 0.0
        while True:
            acc += c[low | R] * a[S ^ (low | R)]
            if R == 0:
                break
            R = (R - 1) & rest
        a[S] = acc
    return a


def run(M4s, n_mat, wt, sigma2, det=False, all_roots=True, want_a=True, n_max=None):
    order = np.array([m.shape[1] for m in M4s], dtype=np.int32)
    moff = B.bipartite_matrix_offsets(order, n_mat)
    flat = np.concatenate([m.ravel() for m in M4s])
    n_max = int(order.max()) if n_max is None else n_max
    d_order = torch.tensor(order, device="cuda")
    d_moff = torch.tensor(moff, device="cuda")
    d_M = torch.tensor(flat, device="cuda")
    per = 1 << n_max
    c = torch.full((len(M4s) * per,), 12345.0, dtype=torch.float64, device="cuda")
    a = torch.full_like(c, 12345.0) if want_a else None
    if det:
        B.cos_connected_det_bipartite_subsets(n_max, d_order, d_moff, sigma2, d_M, c, a, all_roots)
    else:
        B.cos_connected_sum_bipartite_subsets(n_max, d_order, d_moff, n_mat, wt, sigma2, d_M, c, a, all_roots)
    B.cos_sync_status()
    c = c.cpu().numpy().reshape(len(M4s), per)
    return c, (a.cpu().numpy().reshape(len(M4s), per) if want_a else None), (d_order, d_moff, d_M)


def cos_references(M4, sigma2, wt):
    """c(S), mass(S), a(S), amass(S) of every S of one configuration (cycle factors)."""
    n = M4.shape[1]
    Mf = np.repeat(M4, wt, axis=0) if wt > 1 else M4          # loop weight w = w identical flavors
    sf = None if sigma2 is None else np.tile(np.asarray(sigma2), (wt, 1))
    c = np.zeros(1 << n)
    cm = np.zeros(1 << n)
    for S in range(1, 1 << n):
        idx = members(S)
        c[S] = O.bip(sub4(Mf, idx), sf, method="sum_closed", prec="q")
        cm[S] = O.bip(sub4(M4, idx), sigma2, weight=wt, absmode=True, method="sum_dp")
    a = np.zeros(1 << n)
    for s in itertools.product((0, 1), repeat=n):
        Ms, sv = O.bip_assignment(Mf, sf, s)
        _, a_s, _ = O.closed(Ms, sv, prec="q", subsets=True)
        a += np.asarray(a_s)
    a /= np.array([2.0 ** (n - bin(S).count("1")) for S in range(1 << n)])
    a[0] = 1.0
    return c, cm, a, subset_exp(cm, n)


def det_references(G4, alpha2):
    n = G4.shape[1]
    c = np.zeros(1 << n)
    cm = np.zeros(1 << n)
    a = np.zeros(1 << n)
    a[0] = 1.0
    al = np.zeros((2, 2)) if alpha2 is None else np.asarray(alpha2, dtype=np.float64)
    for S in range(1, 1 << n):
        idx = members(S)
        sub = sub4(G4, idx)
        c[S] = O.det_clow(sub, alpha2, prec="q")
        cm[S] = O.det_clow(sub, alpha2, absmode=True)
        tot = 0.0
        for s in itertools.product((0, 1), repeat=len(idx)):
            p = 1.0
            for b in range(2):
                A = np.array([[sub[b, i, s[i], j, s[j]] for j in range(len(idx))] for i in range(len(idx))])
                p *= np.linalg.det(A - np.diag([al[b, s[i]] for i in range(len(idx))]))
            tot += p
        a[S] = tot
    return c, cm, a, subset_exp(cm, n)


def check(c, a, refs, n, k=None):
    cr, cm, ar, am = refs
    assert c[0] == 0.0 and (a is None or a[0] == 1.0)
    for S in range(1, 1 << n):
        sz = bin(S).count("1")
        assert abs(c[S] - cr[S]) <= 64 * sz * EPS64 * cm[S] + 1e-300, (k, S, c[S], cr[S])
        if a is not None:
            assert abs(a[S] - ar[S]) <= 128 * n * EPS64 * am[S] + 1e-300, (k, S, a[S], ar[S])


@pytest.mark.parametrize("n,n_mat,wt,shifts,ncfg", [
    (1, 2, 1, True, 3), (2, 1, 2, False, 4), (3, 2, 1, True, 5), (4, 1, 2, True, 7),
    (5, 2, 1, False, 6), (6, 1, 1, True, 5),
])
def test_bipartite_all_subsets_vs_closed_form(n, n_mat, wt, shifts, ncfg):
    M4s = rand_m4(500 + 10 * n + n_mat, ncfg, n_mat, n)
    sigma2 = np.linspace(-0.2, 0.15, 2 * n_mat).reshape(n_mat, 2).tolist() if shifts else None
    c, a, _ = run(M4s, n_mat, wt, sigma2)
    for k in sorted({0, ncfg // 2, ncfg - 1}):
        check(c[k], a[k], cos_references(M4s[k], sigma2, wt), n, k)


def test_bipartite_uneven_orders_and_padding():
    """Orders 1..6 in one call with n_max = 7: subsets beyond a configuration's order are 0."""
    n_mat = 2
    M4s = [rand_m4(80 + i, 1, n_mat, n)[0] for i, n in enumerate([3, 6, 1, 5, 2, 4, 6])]
    sigma2 = [[0.1, -0.05], [-0.12, 0.07]]
    c, a, _ = run(M4s, n_mat, 1, sigma2, n_max=7)
    for k, M4 in enumerate(M4s):
        n = M4.shape[1]
        assert np.all(c[k][1 << n:] == 0.0) and np.all(a[k][1 << n:] == 0.0)
        if n <= 5:
            check(c[k][:1 << n], a[k][:1 << n], cos_references(M4, sigma2, 1), n, k)


def test_bipartite_root_zero_mode_and_plain_call():
    """all_roots = 0: the subsets containing vertex 0 are the root-0 sweep's own closes, bitwise
    the all-roots values; the rest stays NaN; c(V) is the plain call's output."""
    n, n_mat = 6, 2
    M4s = rand_m4(91, 40, n_mat, n)
    sigma2 = [[0.05, -0.1], [0.08, 0.02]]
    c_all, _, dev = run(M4s, n_mat, 1, sigma2, want_a=False)
    c0, _, _ = run(M4s, n_mat, 1, sigma2, all_roots=False, want_a=False)
    odd = np.arange(1, 1 << n, 2)
    even = np.arange(2, 1 << n, 2)
    assert np.array_equal(c0[:, odd], c_all[:, odd])
    assert np.all(np.isnan(c0[:, even])) and np.all(c0[:, 0] == 0.0)
    out = torch.empty(len(M4s), dtype=torch.float64, device="cuda")
    d_order, d_moff, d_M = dev
    B.cos_connected_sum_bipartite_matrices(n, d_order, d_moff, n_mat, 1, sigma2, d_M, "fp64", out)
    B.cos_sync_status()
    assert np.array_equal(out.cpu().numpy(), c_all[:, (1 << n) - 1])


@pytest.mark.parametrize("n,shifts", [(3, True), (4, False), (5, True)])
def test_det_bipartite_all_subsets(n, shifts):
    G4s = rand_m4(700 + n, 4, 2, n)
    alpha2 = [[0.07, -0.04], [0.03, 0.11]] if shifts else None
    c, a, dev = run(G4s, 2, 1, alpha2, det=True)
    for k in (0, 3):
        check(c[k], a[k], det_references(G4s[k], alpha2), n, k)
    out = torch.empty(len(G4s), dtype=torch.float64, device="cuda")
    d_order, d_moff, d_M = dev
    B.cos_connected_det_bipartite_matrices(n, d_order, d_moff, alpha2, d_M, "fp64", out)
    B.cos_sync_status()
    assert np.array_equal(out.cpu().numpy(), c[:, (1 << n) - 1])


def test_other_precisions_are_rejected():
    M4s = rand_m4(3, 2, 1, 3)
    order = torch.tensor([3, 3], dtype=torch.int32, device="cuda")
    moff = torch.tensor(B.bipartite_matrix_offsets(np.array([3, 3]), 1), device="cuda")
    M = torch.tensor(np.concatenate([m.ravel() for m in M4s]), device="cuda")
    c = torch.empty(2 * 8, dtype=torch.float64, device="cuda")
    lib = B.lib()
    import ctypes
    for prec in ("mixed", "df64"):
        p = B.problem(B.COS_BIPARTITE, B.COS_LOOPS, prec, 3, order, moff=moff, M=M, n_mat=1, loop_weight=1)
        rc = lib.cos_subsets(ctypes.byref(p), 1, B._ptr(c, "f64"), None, None)
        assert rc == -6


def test_honeycomb_workload_order8_sampled():
    """The honeycomb workload at the benchmark's size (2 x 10^4 configurations, SU(2),
    staggered shift, n = 8), determinant weights, in the call the bench times: c(V) equals the
    plain call bitwise; sampled subsets of three configurations against Alg. 1 of the oracle on
    the oracle's own gather."""
    w = I.WORKLOADS["hc_su2_af_n8"]
    nc = w.n_cfg
    cfgs = I.workload_configs(w, nc)
    tabs = B.honeycomb_tables_for(w.model)
    d = B.configs_to_device(cfgs)
    moff = torch.as_tensor(B.bipartite_matrix_offsets(cfgs.order, 2), device="cuda")
    M4 = torch.empty(nc * 2 * 16 * 16, dtype=torch.float64, device="cuda")
    B.cos_gather_bipartite(tabs, *d, moff, M4)
    al = [list(r) for r in w.model.sigma2]
    c = torch.full((nc * 256,), float("nan"), dtype=torch.float64, device="cuda")
    a = torch.full_like(c, float("nan"))
    B.cos_connected_det_bipartite_subsets(8, d[0], moff, al, M4, c, a)
    out = torch.empty(nc, dtype=torch.float64, device="cuda")
    B.cos_connected_det_bipartite_matrices(8, d[0], moff, al, M4, "fp64", out)
    B.cos_sync_status()
    tabs.close()
    c = c.cpu().numpy().reshape(nc, 256)
    a = a.cpu().numpy().reshape(nc, 256)
    assert np.all(np.isfinite(c)) and np.all(np.isfinite(a))
    assert np.array_equal(c[:, 255], out.cpu().numpy())
    otabs = HC.hc_model_tables(w.model)
    rng = np.random.default_rng(8)
    for k in (0, nc // 2, nc - 1):
        o = int(cfgs.offset[k])
        G4 = HC.hc_gather_one(otabs, cfgs.site[o:o + 8], cfgs.tau[o:o + 8], w.model.L, w.model.beta)
        for S in [255, 1, 128] + [int(x) for x in rng.choice(np.arange(2, 255), 8, replace=False)]:
            idx = members(S)
            sub = sub4(G4, idx)
            ref = O.det_clow(sub, al, prec="ld")
            mass = O.det_clow(sub, al, absmode=True)
            assert abs(c[k, S] - ref) <= 64 * len(idx) * EPS64 * mass + 1e-13 * mass, (k, S, c[k, S], ref)
