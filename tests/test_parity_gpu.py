"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances
  * tables, gather: FP64 rounding of the same formula (1e-13 absolute on values <= 1).
  * DP, FP64: relative error <= 1e-10 on the benchmark workloads up to order 8; for
    arbitrary inputs the bound is stated against the absolute mass (sum of |term|
    bound, the same DP on |M|): |err| <= 2^-53 * 64 n * mass, a few ulps per
    visited point of every term.
  * DP, mixed: |err| <= (2n + log2(32 n)) * 2^-24 * mass (FP32 extension; the loop closes
    are compensated FP32-pair dot products, each within gamma_N^2 + 2^-47 of its sum of |terms|
    for N <= n^2 terms, below 1e-9 of the mass at n = 12, which the 2^-24 terms dominate).
  * DP, df64 (FP32 pairs, compensated dot products): |err| <= (16 n^2 + 64 n) * 2^-48 * mass.
    Per dot product of K <= n terms: the matrices' df64 split (2^-48 relative), the FP32
    error accumulator c (of size <= 3K 2^-24 sum|terms|) rounded K times (3K 2^-48), and the
    dropped lo*lo cross terms, whose state part is c of the previous layer (3K 2^-48
    relative to the mass): together <= (7K + 2) 2^-48 sum|terms|.  The 2n layers add these
    relative to the mass; the flavor sums and seeds (df64 additions, <= 2^-45 of their
    operands' magnitudes) add at most 32 n 2^-48.
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
# Error measures: 1e-10 relative for kappa = mass / |c| <= 1e5; above, the mass-relative bound.
KAPPA_RELATIVE_TARGET = 1e5
# Entrywise agreement of the GPU's and the oracle's propagator matrices (independent tables).
TABLE_ABS = 1e-13


def fp64_bound(n, mass):
    return 64 * n * EPS64 * mass


def mixed_bound(n, mass):
    return (2 * n + math.log2(32 * n)) * EPS32 * mass


def df64_bound(n, mass):
    return (16 * n * n + 64 * n) * 2.0 ** -48 * mass


def run_matrices(Ms_list, n_mat, loop_weight, sigma, precision="fp64", abs_mass=False):
    """Pack per-configuration matrices [n_mat][n][n] (uneven n allowed) and run the DP."""
    order = np.array([m.shape[-1] for m in Ms_list], dtype=np.int32)
    moff = B.matrix_offsets(order, n_mat)
    flat = np.concatenate([np.asarray(m, dtype=np.float64).ravel() for m in Ms_list]) if Ms_list else np.zeros(1)
    d_order = torch.tensor(order, device="cuda")
    d_moff = torch.tensor(moff, device="cuda")
    d_M = torch.tensor(flat, device="cuda")
    out = torch.full((len(Ms_list),), float("nan"), dtype=torch.float64, device="cuda")
    mass = torch.full_like(out, float("nan")) if abs_mass else None
    n_max = int(order.max()) if len(order) else 1
    B.cos_connected_sum_matrices(n_max, d_order, d_moff, n_mat, loop_weight, sigma, d_M, precision, out, mass)
    B.cos_sync_status()
    return out.cpu().numpy(), (mass.cpu().numpy() if abs_mass else None)


def rand_mats(seed, ncfg, nf, n, scale=0.9):
    return list(I.random_matrices(seed, ncfg, nf, n, scale))


# ------------------------------------------------------------------ K-TAB / K-GATHER

@pytest.mark.parametrize("name", ["su2_sym_n4", "su4_mu_broken_n8", "su3_shift_mixed_n10", "su6_sym_uneven_n4_12"])
def test_tables_match_oracle(name):
    model = I.WORKLOADS[name].model
    tabs = B.tables_for(model)
    got = tabs.table().cpu().numpy()
    ref = P.model_tables(model)
    if model.symmetric:
        ref = ref[:1]
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) < 1e-13
    inf = tabs.info()
    assert inf.symmetric == int(model.symmetric)
    assert np.allclose(list(inf.sigma)[:inf.n_mat], list(model.sigma)[:inf.n_mat])
    tabs.close()


def test_dmu_table_matches_oracle():
    model = I.WORKLOADS["su4_adjoint_n10"].model
    tabs = B.tables_for(model)
    got = tabs.table(deriv=True).cpu().numpy()
    ref = P.model_tables(model, deriv=True)
    assert np.max(np.abs(got - ref)) < 1e-12
    tabs.close()


def test_gather_matches_oracle_uneven():
    w = I.WORKLOADS["su6_sym_uneven_n4_12"]
    cfgs = I.workload_configs(w, 45)
    model = I.Model(w.model.L, 1.0, w.model.beta, 1.0, (0.1, -0.3), (0.05, 0.0), w.model.n_tau)  # broken, 2 flavors
    tabs = B.tables_for(model)
    d = B.configs_to_device(cfgs)
    moff = B.matrix_offsets(cfgs.order, 2)
    M = torch.zeros(int(moff[-1] + 2 * cfgs.order[-1] ** 2), dtype=torch.float64, device="cuda")
    B.cos_gather(tabs, *d, torch.tensor(moff, device="cuda"), M)
    B.cos_sync_status()
    got = M.cpu().numpy()
    ref = P.gather(P.model_tables(model), cfgs, model.L, model.beta)
    for c in range(cfgs.n_cfg):
        n = cfgs.order[c]
        blk = got[moff[c]:moff[c] + 2 * n * n].reshape(2, n, n)
        assert np.max(np.abs(blk - ref[c])) < 1e-13, c
    tabs.close()


def test_gather_flags_bad_site():
    model = I.WORKLOADS["su2_sym_n4"].model
    tabs = B.tables_for(model)
    cfgs = I.workload_configs(I.WORKLOADS["su2_sym_n4"], 3)
    cfgs.site[5] = model.L * model.L          # out of range
    d = B.configs_to_device(cfgs)
    M = torch.zeros(3 * 16, dtype=torch.float64, device="cuda")
    B.cos_gather(tabs, *d, torch.arange(3, dtype=torch.int64, device="cuda") * 16, M)
    with pytest.raises(B.CosError) as ei:
        B.cos_sync_status()
    assert ei.value.status == -1
    B.cos_sync_status()                      # the status word was cleared
    tabs.close()


# ------------------------------------------------------------------ K-DP from matrices

CASES = [  # n, n_mat, loop_weight, shifts, ncfg
    (1, 1, 2, False, 5), (1, 3, 1, True, 7), (2, 2, 1, True, 33), (3, 1, 6, False, 40),
    (4, 4, 1, False, 70), (4, 3, 1, True, 21), (5, 1, 4, True, 65), (6, 2, 1, True, 19),
    (7, 5, 1, False, 9), (8, 4, 1, False, 17), (8, 1, 3, False, 35), (9, 3, 1, True, 4),
]


@pytest.mark.parametrize("n,n_mat,wt,shifts,ncfg", CASES)
def test_dp_fp64_matches_oracle(n, n_mat, wt, shifts, ncfg):
    Ms = rand_mats(100 + n * 7 + n_mat, ncfg, n_mat, n)
    sig = list(np.linspace(-0.2, 0.15, n_mat)) if shifts else None
    got, mass = run_matrices(Ms, n_mat, wt, sig, abs_mass=True)
    for c in range(ncfg):
        ref = O.dp(Ms[c], sig, weight=wt, prec="ld")
        rmass = O.dp(Ms[c], sig, weight=wt, absmode=True)
        assert abs(got[c] - ref) <= fp64_bound(n, rmass), (c, got[c], ref, rmass)
        assert mass[c] == pytest.approx(rmass, rel=1e-12)


@pytest.mark.parametrize("n,n_mat,wt,shifts,ncfg", [(4, 3, 1, True, 40), (6, 1, 6, False, 33), (8, 4, 1, True, 12),
                                                   (10, 3, 1, True, 3)])
def test_dp_mixed_within_bound(n, n_mat, wt, shifts, ncfg):
    Ms = rand_mats(300 + n, ncfg, n_mat, n)
    sig = list(np.linspace(-0.1, 0.1, n_mat)) if shifts else None
    got, _ = run_matrices(Ms, n_mat, wt, sig, precision="mixed")
    for c in range(ncfg):
        ref = O.dp(Ms[c], sig, weight=wt, prec="ld")
        rmass = O.dp(Ms[c], sig, weight=wt, absmode=True)
        assert abs(got[c] - ref) <= mixed_bound(n, rmass), (c, got[c], ref, rmass)


@pytest.mark.parametrize("n,n_mat,wt,shifts,ncfg", CASES)
def test_dp_df64_matches_oracle(n, n_mat, wt, shifts, ncfg):
    Ms = rand_mats(700 + n * 7 + n_mat, ncfg, n_mat, n)
    sig = list(np.linspace(-0.2, 0.15, n_mat)) if shifts else None
    got, mass = run_matrices(Ms, n_mat, wt, sig, precision="df64", abs_mass=True)
    for c in range(ncfg):
        ref = O.dp(Ms[c], sig, weight=wt, prec="ld")
        rmass = O.dp(Ms[c], sig, weight=wt, absmode=True)
        assert abs(got[c] - ref) <= df64_bound(n, rmass), (c, got[c], ref, rmass)
        assert abs(mass[c] - rmass) <= df64_bound(n, rmass), (c, mass[c], rmass)


def test_dp_df64_uneven_orders_and_max_order():
    """Orders 1..12 in one launch (order 12 at the structure's largest layers); the order-12
    configurations are checked against the oracle in double, whose own error is far below
    the df64 bound at this mass."""
    rng = np.random.default_rng(8)
    orders = rng.integers(1, 10, size=80)
    orders[:3] = [12, 11, 10]
    Ms = [I.random_matrices(int(2000 + c), 1, 3, int(n), 0.9)[0] for c, n in enumerate(orders)]
    sig = [0.07, 0.0, -0.11]
    got, _ = run_matrices(Ms, 3, 1, sig, precision="df64")
    for c in list(range(3)) + list(range(3, 80, 9)):
        ref = O.dp(Ms[c], sig, prec="ld" if orders[c] <= 10 else "d")
        rmass = O.dp(Ms[c], sig, absmode=True)
        assert abs(got[c] - ref) <= df64_bound(int(orders[c]), rmass), (c, orders[c], got[c], ref)


def test_dp_uneven_orders_one_launch():
    rng = np.random.default_rng(5)
    orders = rng.integers(1, 10, size=150)
    orders[:3] = [12, 11, 10]
    Ms = [I.random_matrices(int(1000 + c), 1, 2, int(n), 0.9)[0] for c, n in enumerate(orders)]
    got, _ = run_matrices(Ms, 2, 1, [0.05, -0.12])
    for c in list(range(3)) + list(range(3, 150, 7)):
        ref = O.dp(Ms[c], [0.05, -0.12], prec="d")
        rmass = O.dp(Ms[c], [0.05, -0.12], absmode=True)
        assert abs(got[c] - ref) <= fp64_bound(int(orders[c]), rmass), (c, orders[c])


def test_dp_empty_and_deterministic():
    got, _ = run_matrices([], 1, 2, None)
    assert got.shape == (0,)
    Ms = rand_mats(9, 50, 3, 7)
    a, _ = run_matrices(Ms, 3, 1, [0.1, 0.2, 0.3])
    b, _ = run_matrices(Ms, 3, 1, [0.1, 0.2, 0.3])
    assert np.array_equal(a, b)


def test_dp_rejects_orders_above_nmax():
    Ms = rand_mats(2, 4, 1, 5)
    order = torch.tensor([5, 5, 6, 5], dtype=torch.int32, device="cuda")     # 6 > n_max = 5
    moff = torch.arange(4, dtype=torch.int64, device="cuda") * 25
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    B.cos_connected_sum_matrices(5, order, moff, 1, 2, None, torch.tensor(np.stack(Ms).ravel(), device="cuda"),
                                 "fp64", out)
    with pytest.raises(B.CosError) as ei:
        B.cos_sync_status()
    assert ei.value.status == -2


def test_dp_order12_relabel_invariance():
    """At full size no oracle is cheap; vertex relabeling (head rule) and the
    transpose must leave c unchanged, and the oracle checks one sample."""
    M = I.random_matrices(77, 1, 1, 12, 0.9)[0]
    perm = np.random.default_rng(1).permutation(12)
    Mp = M[:, perm][:, :, perm]
    got, mass = run_matrices([M, Mp, M.transpose(0, 2, 1)], 1, 6, None, abs_mass=True)
    assert abs(got[1] - got[0]) <= fp64_bound(12, mass[0])
    assert abs(got[2] - got[0]) <= fp64_bound(12, mass[0])
    ref = O.dp(M, None, weight=6, prec="d")
    assert abs(got[0] - ref) <= fp64_bound(12, mass[0])


@pytest.mark.parametrize("precision", ["mixed", "df64"])
def test_order11_invariances_reduced_precision(precision):
    """Relabeling and transpose at order 11 with three broken flavors and shifts, for the
    reduced-precision kernels (two and four configurations per lane): each result stays
    within its mode's bound of the FP64 one."""
    n, nf = 11, 3
    M = I.random_matrices(88, 1, nf, n, 0.9)[0]
    perm = np.random.default_rng(2).permutation(n)
    Ms = [M, M[:, perm][:, :, perm], M.transpose(0, 2, 1)] * 3   # several per batch
    sig = [0.08, -0.05, 0.0]
    ref, mass = run_matrices(Ms, nf, 1, sig, abs_mass=True)
    got, _ = run_matrices(Ms, nf, 1, sig, precision=precision)
    bound = mixed_bound(n, mass[0]) if precision == "mixed" else df64_bound(n, mass[0])
    assert np.all(np.abs(ref - ref[0]) <= fp64_bound(n, mass[0]))
    assert np.all(np.abs(got - ref[0]) <= bound + fp64_bound(n, mass[0]))


# ------------------------------------------------------------------ workloads through the coordinates path

def workload_check(name, n_cfg, sample, prec="fp64", rel=1e-10, graph=False):
    """The workload at the benchmark's size and launch form (graph=True: the CUDA-graph plan
    the benchmark replays), sampled configurations against the oracle.

    Per configuration:
      * the inputs: the GPU gather's matrices equal the oracle's (its own tables, its own
        gather) within TABLE_ABS entry by entry (two independent momentum sums differ by
        rounding);
      * the DP on identical inputs: the oracle DP (long double) on the GPU's matrices against
        the GPU result, within the precision's bound (and 1e-10 relative in FP64 for
        kappa <= 1e5);
      * end to end, against the oracle DP on its own matrices: every term is a product of
        entries, so an entrywise input difference <= delta moves c by at most
        mass(|M| + delta) - mass(|M|) (the absolute-value DP is monotone in every entry);
        the GPU result lies within that plus the DP bound."""
    w = I.WORKLOADS[name]
    n_cfg = w.n_cfg if n_cfg is None else n_cfg
    cfgs = I.workload_configs(w, n_cfg)
    tabs = B.tables_for(w.model)
    d = B.configs_to_device(cfgs)
    out = torch.full((n_cfg,), float("nan"), dtype=torch.float64, device="cuda")
    mass = torch.full_like(out, float("nan"))
    nmax = int(cfgs.order.max())
    B.cos_connected_sum_batch(tabs, nmax, *d, prec, mass.new_empty(n_cfg), mass)   # the mass (plain call)
    if graph:
        plan = B.cos_plan_create_batch(tabs, nmax, *d, prec, out)
        out.fill_(float("nan"))
        plan.launch()
        plan.status()
        plan.close()
    else:
        B.cos_connected_sum_batch(tabs, nmax, *d, prec, out)
    n_mat = tabs.info().n_mat
    moff = B.matrix_offsets(cfgs.order, n_mat)
    gM = torch.empty(int(n_mat * (cfgs.order.astype(np.int64) ** 2).sum()), dtype=torch.float64, device="cuda")
    B.cos_gather(tabs, *d, torch.as_tensor(moff, device="cuda"), gM)
    B.cos_sync_status()
    got, gmass, gmat = out.cpu().numpy(), mass.cpu().numpy(), gM.cpu().numpy()
    otabs = P.model_tables(w.model)
    wt = 1
    sig = list(w.model.sigma)
    if w.model.symmetric:
        otabs, wt, sig = otabs[:1], w.model.n_flavors, sig[:1]
    if not any(sig):
        sig = None
    bound = {"fp64": fp64_bound, "df64": df64_bound, "mixed": mixed_bound}[prec]
    idx = sorted(set(np.linspace(0, n_cfg - 1, sample).astype(int)))
    errs = []
    for c, M in zip(idx, P.gather(otabs, cfgs, w.model.L, w.model.beta, idx)):
        n = int(cfgs.order[c])
        Mg = gmat[moff[c]:moff[c] + n_mat * n * n].reshape(n_mat, n, n)
        ref_g = O.dp(Mg, sig, weight=wt, prec="ld")          # identical inputs
        ref_o = O.dp(M, sig, weight=wt, prec="ld")           # the oracle's own tables
        rmass = O.dp(Mg, sig, weight=wt, absmode=True)
        assert gmass[c] == pytest.approx(rmass, rel=1e-10 if prec != "mixed" else 1e-5)
        e = abs(got[c] - ref_g)
        tol = bound(n, rmass)
        if prec == "fp64":
            tol = max(rel * abs(ref_g), tol)
            # the relative target holds for condition numbers kappa = mass / |c| up to 1e5;
            # beyond that the mass-relative bound is the statement
            if rmass / abs(ref_g) <= KAPPA_RELATIVE_TARGET:
                errs.append(e / abs(ref_g))
        assert e <= tol, (c, n, got[c], ref_g, rmass)
        assert np.max(np.abs(Mg - M)) <= TABLE_ABS, (c, np.max(np.abs(Mg - M)))
        grow = O.dp(np.abs(Mg) + TABLE_ABS, None if sig is None else np.abs(sig), weight=wt, absmode=True,
                    prec="ld") - O.dp(np.abs(Mg), None if sig is None else np.abs(sig), weight=wt, absmode=True,
                                      prec="ld")
        assert abs(got[c] - ref_o) <= grow + tol, (c, n, got[c], ref_o, grow, tol)
    tabs.close()
    return errs


def test_workload_su2_order4_all_configs():
    n_cfg = I.WORKLOADS["su2_sym_n4"].n_cfg
    errs = workload_check("su2_sym_n4", None, n_cfg)
    assert len(errs) >= n_cfg - 10        # every configuration checked; 4 have kappa > 1e5
    assert max(errs) < 1e-10


def test_workload_su4_order8_sampled():
    errs = workload_check("su4_mu_broken_n8", None, 40)
    assert max(errs) < 1e-10


def test_workload_su3_mixed_order10_sampled():
    workload_check("su3_shift_mixed_n10", None, 6, prec="mixed")


def test_workload_su3_fp64_order10_sampled():
    workload_check("su3_shift_mixed_n10", None, 4, prec="fp64")


def test_workload_su6_uneven_sampled():
    workload_check("su6_sym_uneven_n4_12", None, 12, graph=True)


def test_workload_su4_df64_order8_sampled():
    workload_check("su4_mu_broken_n8", None, 40, prec="df64")


def test_workload_su3_df64_order10_sampled():
    workload_check("su3_shift_mixed_n10", None, 4, prec="df64")


def test_workload_su6_uneven_df64_sampled():
    workload_check("su6_sym_uneven_n4_12", None, 10, prec="df64")


def test_workload_su4_mixed_order8_sampled():
    workload_check("su4_mu_broken_n8", None, 12, prec="mixed")
