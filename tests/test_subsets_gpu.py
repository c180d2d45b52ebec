"""GPU parity of the all-subsets mode (cos_connected_sum_subsets) against the oracle.

References (none of them runs the merged DP), in __float128: the closed form's subset
subtraction cancels a(S) ~ 10 against c(S) ~ 1e-7 on the order-8 workload, so long double
would not resolve the FP64 DP's mass-relative error.
  * c(S): the oracle's closed form (tier 1: determinants + the subset recursion of Methods A)
    on the principal submatrices M^l[S, S], one call per subset S.
  * a(S): the same closed form's sum over all decorated covers of S (flavor DP over
    determinants), so the GPU subset exponential a = sum c(T) a(S \\ T) is checked against a
    route that never forms c.
Tolerances, per subset, against the absolute mass (the same DP on |M|, |sigma|: a bound on the
sum of |term| of c(S)), and amass = the subset exponential of the masses (bound for a(S)):
  FP64  |c err| <= 64 |S| 2^-53 mass(S),          |a err| <= 128 n 2^-53 amass(S)
  mixed |c err| <= (2|S| + log2(32|S|)) 2^-24 mass(S),  |a err| <= twice that with amass.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from oracle import propagators as P
from paper_2507_12349_b300 import binding as B
from paper_2507_12349_b300 import inputs as I

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24


def members(S):
    return [i for i in range(S.bit_length()) if S >> i & 1]


def run_subsets(Ms, n_mat, wt, sigma, precision="fp64", all_roots=True, want_a=True, n_max=None):
    order = np.array([m.shape[-1] for m in Ms], dtype=np.int32)
    moff = B.matrix_offsets(order, n_mat)
    flat = np.concatenate([np.asarray(m, dtype=np.float64).ravel() for m in Ms])
    n_max = int(order.max()) if n_max is None else n_max
    d_order = torch.tensor(order, device="cuda")
    d_moff = torch.tensor(moff, device="cuda")
    d_M = torch.tensor(flat, device="cuda")
    per = 1 << n_max
    c = torch.full((len(Ms) * per,), 12345.0, dtype=torch.float64, device="cuda")
    a = torch.full_like(c, 12345.0) if want_a else None
    B.cos_connected_sum_subsets(n_max, d_order, d_moff, n_mat, wt, sigma, d_M, precision, c, a, all_roots)
    B.cos_sync_status()
    c = c.cpu().numpy().reshape(len(Ms), per)
    return c, (a.cpu().numpy().reshape(len(Ms), per) if want_a else None), (d_order, d_moff, d_M)


def flavors(M, sigma, wt):
    """Loop weight w as w identical flavors (each loop's flavor sum then gives w)."""
    if wt == 1:
        return M, sigma
    return np.repeat(M, wt, axis=0), (None if sigma is None else list(sigma) * wt)


def references(M, sigma, wt):
    """c(S), a(S) and their masses for every S of one configuration, from the oracle."""
    n = M.shape[-1]
    Mf, sf = flavors(M, sigma, wt)
    c = np.zeros(1 << n)
    cm = np.zeros(1 << n)
    for S in range(1, 1 << n):
        idx = members(S)
        sub = Mf[:, idx][:, :, idx]
        c[S] = O.closed(sub, sf, prec="q")
        cm[S] = O.dp(M[:, idx][:, :, idx], sigma, weight=wt, absmode=True)
    _, a, c0 = O.closed(Mf, sf, prec="q", subsets=True)
    am = np.zeros(1 << n)
    am[0] = 1.0
    for S in range(1, 1 << n):
        low = S & -S
        rest = S ^ low
        R = rest
        acc = 0.0
        while True:
            acc += cm[low | R] * am[S ^ (low | R)]
            if R == 0:
                break
            R = (R - 1) & rest
        am[S] = acc
    # the oracle's own subset recursion agrees with the per-subset closed forms (S containing 0)
    odd = np.arange(1, 1 << n, 2)
    assert np.allclose(c0[odd], c[odd], rtol=1e-9, atol=1e-12 * np.max(cm))
    return c, cm, a, am


def bounds(S_size, mass, precision, n):
    if precision == "fp64":
        return 64 * max(S_size, 1) * EPS64 * mass
    return (2 * S_size + math.log2(32 * max(S_size, 1))) * EPS32 * mass


@pytest.mark.parametrize("n,n_mat,wt,shifts,ncfg,precision", [
    (1, 3, 1, True, 4, "fp64"), (2, 2, 1, False, 5, "fp64"), (3, 1, 3, True, 7, "fp64"),
    (4, 3, 1, True, 9, "fp64"), (5, 2, 1, False, 6, "fp64"), (6, 4, 1, False, 9, "fp64"),
    (6, 2, 1, True, 17, "fp64"), (5, 3, 1, True, 11, "mixed"), (6, 1, 6, False, 7, "mixed"),
])
def test_all_subsets_vs_closed_form(n, n_mat, wt, shifts, ncfg, precision):
    Ms = list(I.random_matrices(900 + 10 * n + n_mat, ncfg, n_mat, n, 0.9))
    sigma = list(np.linspace(-0.2, 0.15, n_mat)) if shifts else None
    c, a, _ = run_subsets(Ms, n_mat, wt, sigma, precision)
    for k in sorted({0, ncfg // 2, ncfg - 1}):
        cr, cm, ar, am = references(Ms[k], sigma, wt)
        assert c[k][0] == 0.0 and a[k][0] == 1.0
        for S in range(1, 1 << n):
            sz = bin(S).count("1")
            assert abs(c[k][S] - cr[S]) <= bounds(sz, cm[S], precision, n) + 1e-300, (k, S, c[k][S], cr[S])
            assert abs(a[k][S] - ar[S]) <= 2 * bounds(n, am[S], precision, n) + 1e-300, (k, S, a[k][S], ar[S])


def test_uneven_orders_and_padding():
    """Orders 1..7 in one call with n_max = 8: sets beyond a configuration's order are 0."""
    rng = np.random.default_rng(5)
    n_mat = 2
    Ms = [I.random_matrices(70 + i, 1, n_mat, n, 0.9)[0] for i, n in enumerate([3, 7, 1, 5, 2, 6, 4, 7])]
    sigma = [0.1, -0.12]
    c, a, _ = run_subsets(Ms, n_mat, 1, sigma, n_max=8)
    for k, M in enumerate(Ms):
        n = M.shape[-1]
        assert np.all(c[k][1 << n:] == 0.0) and np.all(a[k][1 << n:] == 0.0)
        cr, cm, ar, am = references(M, sigma, 1)
        for S in rng.choice(np.arange(1, 1 << n), size=min(12, (1 << n) - 1), replace=False):
            S = int(S)
            assert abs(c[k][S] - cr[S]) <= bounds(bin(S).count("1"), cm[S], "fp64", n), (k, S)
            assert abs(a[k][S] - ar[S]) <= 2 * bounds(n, am[S], "fp64", n), (k, S)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
def test_root_zero_mode_is_the_dp_by_product(precision):
    """all_roots = 0: sets holding vertex 0 equal the all-roots values bit for bit (same per-lane
    arithmetic), the other sets are NaN, and c(V) equals cos_connected_sum_matrices."""
    n, n_mat = 7, 3
    Ms = list(I.random_matrices(31, 40, n_mat, n, 0.9))
    sigma = [0.05, 0.0, -0.1]
    c0, _, dev = run_subsets(Ms, n_mat, 1, sigma, precision, all_roots=False, want_a=False)
    c1, _, _ = run_subsets(Ms, n_mat, 1, sigma, precision, all_roots=True, want_a=False)
    odd = np.arange(1, 1 << n, 2)
    even = np.arange(2, 1 << n, 2)
    assert np.array_equal(c0[:, odd], c1[:, odd])
    assert np.all(np.isnan(c0[:, even])) and np.all(c0[:, 0] == 0.0)
    assert not np.any(np.isnan(c1))
    d_order, d_moff, d_M = dev
    out = torch.empty(40, dtype=torch.float64, device="cuda")
    B.cos_connected_sum_matrices(n, d_order, d_moff, n_mat, 1, sigma, d_M, precision, out)
    B.cos_sync_status()
    assert np.array_equal(out.cpu().numpy(), c1[:, (1 << n) - 1])


def test_order8_workload_all_subsets():
    """SU(4), mu broken, n = 8 (the benchmark's configurations): every subset of two of them."""
    w = I.WORKLOADS["su4_mu_broken_n8"]
    cfgs = I.workload_configs(w, 48)
    otabs = P.model_tables(w.model)
    Ms = []
    for k in range(48):
        o = int(cfgs.offset[k])
        Ms.append(P.gather_one(otabs, cfgs.site[o:o + 8], cfgs.tau[o:o + 8], w.model.L, w.model.beta))
    c, a, _ = run_subsets(Ms, 4, 1, None)
    for k in (0, 47):
        cr, cm, ar, am = references(Ms[k], None, 1)
        for S in range(1, 256):
            sz = bin(S).count("1")
            assert abs(c[k][S] - cr[S]) <= bounds(sz, cm[S], "fp64", 8), (k, S, c[k][S], cr[S])
            assert abs(a[k][S] - ar[S]) <= 2 * bounds(8, am[S], "fp64", 8), (k, S, a[k][S], ar[S])
