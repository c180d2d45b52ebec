"""GPU parity of the bipartite (two-sublattice) path against the oracle.

The oracle value is the definition: the sum over every sublattice assignment of the merged DP
(`oracle.bip(..., method="sum_dp")`, long double), itself pinned against the closed form,
brute force and the sublattice-resolved DP of Alg. 1-2 in test_oracle_bip_pins.
Tolerance: |err| <= 64 n 2^-53 mass, the FP64 bound of the square-lattice tests; the mass
(the same DP on |M4|, |sigma| with all signs +) sums the assignments' masses.
"""
import functools
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from oracle import honeycomb as HC
from paper_2507_12349_b300 import autograd as AG
from paper_2507_12349_b300 import binding as B
from paper_2507_12349_b300 import inputs as I

pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53


def bound(n, mass):
    return 64 * n * EPS64 * mass


def rand_m4(seed, ncfg, nf, n, scale=0.9):
    M = I.random_matrices(seed, ncfg, nf, 2 * n, scale)         # [cfg][nf][2n][2n], index i*2 + s
    return [np.ascontiguousarray(m.reshape(nf, n, 2, n, 2)) for m in M]


def df64_bound(n, mass):
    return (16 * n * n + 64 * n) * 2.0 ** -48 * mass


def mixed_bound(n, mass):
    """FP32 extension, FP64 close: a few FP32 ulps per visited point of every term (2n), and
    the rounding of dot products of up to 2n - 1 states (log2 of the fan-in)."""
    return (2 * n + math.log2(64 * n)) * 2.0 ** -24 * mass


def run(M4s, n_mat, wt, sigma2, abs_mass=False, n_max=None, precision="fp64"):
    order = np.array([m.shape[1] for m in M4s], dtype=np.int32)
    moff = B.bipartite_matrix_offsets(order, n_mat)
    flat = np.concatenate([m.ravel() for m in M4s])
    d_order = torch.tensor(order, device="cuda")
    d_moff = torch.tensor(moff, device="cuda")
    d_M = torch.tensor(flat, device="cuda")
    out = torch.full((len(M4s),), float("nan"), dtype=torch.float64, device="cuda")
    mass = torch.full_like(out, float("nan")) if abs_mass else None
    n_max = int(order.max()) if n_max is None else n_max
    B.cos_connected_sum_bipartite_matrices(n_max, d_order, d_moff, n_mat, wt, sigma2, d_M, precision, out, mass)
    B.cos_sync_status()
    return out.cpu().numpy(), (mass.cpu().numpy() if abs_mass else None)


CASES = [  # n, n_mat, loop weight, shifts, configurations
    (1, 2, 1, True, 5), (2, 1, 2, False, 9), (3, 2, 1, True, 17), (4, 1, 3, True, 33), (4, 3, 1, False, 7),
    (5, 2, 1, True, 12), (6, 1, 2, True, 6), (7, 2, 1, False, 3),
]


@pytest.mark.parametrize("n,n_mat,wt,shifts,ncfg", CASES)
def test_bipartite_matches_oracle(n, n_mat, wt, shifts, ncfg):
    M4s = rand_m4(500 + 10 * n + n_mat, ncfg, n_mat, n)
    s2 = np.array([[0.11 - 0.05 * l, -0.07 + 0.04 * l] for l in range(n_mat)]) if shifts else None
    got, mass = run(M4s, n_mat, wt, None if s2 is None else s2.tolist(), abs_mass=True)
    for c in sorted({0, ncfg // 2, ncfg - 1}):
        ref = O.bip(M4s[c], s2, weight=wt, method="sum_dp", prec="ld")
        rmass = O.bip(M4s[c], s2, weight=wt, method="sum_dp", absmode=True)
        assert abs(got[c] - ref) <= bound(n, rmass), (c, got[c], ref, rmass)
        assert mass[c] == pytest.approx(rmass, rel=1e-12)


@pytest.mark.parametrize("n,n_mat,wt,shifts,ncfg", CASES[1::2])
def test_bipartite_df64_matches_oracle(n, n_mat, wt, shifts, ncfg):
    M4s = rand_m4(800 + 10 * n + n_mat, ncfg, n_mat, n)
    s2 = np.array([[0.09 - 0.04 * l, -0.06 + 0.05 * l] for l in range(n_mat)]) if shifts else None
    got, mass = run(M4s, n_mat, wt, None if s2 is None else s2.tolist(), abs_mass=True, precision="df64")
    for c in sorted({0, ncfg // 2, ncfg - 1}):
        ref = O.bip(M4s[c], s2, weight=wt, method="sum_dp", prec="ld")
        rmass = O.bip(M4s[c], s2, weight=wt, method="sum_dp", absmode=True)
        assert abs(got[c] - ref) <= df64_bound(n, rmass), (c, got[c], ref, rmass)
        assert abs(mass[c] - rmass) <= df64_bound(n, rmass)


@pytest.mark.parametrize("n,n_mat,wt,shifts,ncfg", CASES[::2])
def test_bipartite_mixed_matches_oracle(n, n_mat, wt, shifts, ncfg):
    M4s = rand_m4(600 + 10 * n + n_mat, ncfg, n_mat, n)
    s2 = np.array([[0.1 - 0.03 * l, -0.05 + 0.02 * l] for l in range(n_mat)]) if shifts else None
    got, mass = run(M4s, n_mat, wt, None if s2 is None else s2.tolist(), abs_mass=True, precision="mixed")
    for c in sorted({0, ncfg // 2, ncfg - 1}):
        ref = O.bip(M4s[c], s2, weight=wt, method="sum_dp", prec="ld")
        rmass = O.bip(M4s[c], s2, weight=wt, method="sum_dp", absmode=True)
        assert abs(got[c] - ref) <= mixed_bound(n, rmass), (c, got[c], ref, rmass)
        assert mass[c] == pytest.approx(rmass, rel=1e-5)


UNEVEN_ORDERS = [9, 3, 8, 1, 6, 2, 7, 5, 4, 9]
UNEVEN_SIG = [0.06, -0.09]


@functools.lru_cache(maxsize=1)
def uneven_case():
    """Orders 1..9 for one launch, with the oracle's value and mass of each configuration.  At
    n = 9 (512 assignments) the equal-block identity gives the reference: every assignment sees
    the same matrices, so c_bip = 2^9 c."""
    M4s, refs = [], []
    s2 = [[UNEVEN_SIG[0], UNEVEN_SIG[0]], [UNEVEN_SIG[1], UNEVEN_SIG[1]]]
    for c, n in enumerate(UNEVEN_ORDERS):
        if n == 9:
            M = I.random_matrices(900 + c, 1, 2, n, 0.9)[0]
            M4s.append(np.ascontiguousarray(np.broadcast_to(M[:, :, None, :, None], (2, n, 2, n, 2))))
            refs.append((2 ** 9 * O.dp(M, UNEVEN_SIG, prec="ld"), 2 ** 9 * O.dp(M, UNEVEN_SIG, absmode=True)))
        else:
            M4s.append(rand_m4(700 + c, 1, 2, n)[0])
            refs.append((O.bip(M4s[-1], np.array(s2), method="sum_dp", prec="ld"),
                         O.bip(M4s[-1], np.array(s2), method="sum_dp", absmode=True)))
    return M4s, s2, refs


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
def test_bipartite_uneven_orders_and_order9(precision):
    """Orders 1..9 in one launch, in every precision (the rows' state masks reach bit 2n + 1)."""
    M4s, s2, refs = uneven_case()
    got, mass = run(M4s, 2, 1, s2, abs_mass=True, precision=precision)
    tol = {"fp64": bound, "mixed": mixed_bound, "df64": df64_bound}[precision]
    for c, n in enumerate(UNEVEN_ORDERS):
        ref, rmass = refs[c]
        assert abs(got[c] - ref) <= tol(n, rmass), (c, n, got[c], ref)
        assert mass[c] == pytest.approx(rmass, rel=1e-5 if precision == "mixed" else 1e-12)


@pytest.mark.parametrize("precision", ["mixed", "df64"])
@pytest.mark.parametrize("n_mat,wt", [(1, 1), (2, 1), (3, 2)])
def test_bipartite_two_per_lane_bitwise(precision, n_mat, wt):
    """Mixed mode, and double-float at loop weight 1, run two configurations per lane up to
    n_max = 8 and one per lane at n_max = 9, on the same configurations (uneven orders; batches
    whose lanes hold one or two configurations).  Double-float: each packed operation is the
    one-per-lane operation and the close's sign is applied after the flavor sum (exact, every
    compensated step being symmetric under negation), so both give the same values.  Mixed:
    the extensions are the same operations, but two per lane close with compensated FP32 sums
    (about 47 bits) where one per lane closes in FP64, and a seed rounded to FP32 may then
    differ by an ulp; the two agree within the mixed mode's error bound."""
    orders = [8, 3, 7, 1, 6, 5, 8, 2, 4] + [5] * 41 + [7] * 3
    M4s = [rand_m4(9900 + c, 1, n_mat, n)[0] for c, n in enumerate(orders)]
    s2 = [[0.05 - 0.02 * l, -0.03 + 0.01 * l] for l in range(n_mat)]
    a, ma = run(M4s, n_mat, wt, s2, abs_mass=True, precision=precision)
    b, mb = run(M4s, n_mat, wt, s2, abs_mass=True, precision=precision, n_max=9)
    assert np.all(np.isfinite(a))
    if precision == "df64":
        assert np.array_equal(a, b) and np.array_equal(ma, mb)
    else:
        for c, n in enumerate(orders):
            assert abs(a[c] - b[c]) <= mixed_bound(n, mb[c]), (c, n, a[c], b[c])
            assert ma[c] == pytest.approx(mb[c], rel=1e-5)


@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64"])
def test_bipartite_empty_batch_and_order_above_nmax(precision):
    """No configurations: nothing to do, nothing written.  An order above n_max: the planner
    flags it (COS_ERR_ORDER at the next status read), in every precision's sweep (two
    configurations per lane in mixed and double-float at n_max <= 8)."""
    empty_i = torch.zeros(0, dtype=torch.int32, device="cuda")
    out = torch.zeros(0, dtype=torch.float64, device="cuda")
    B.cos_connected_sum_bipartite_matrices(4, empty_i, torch.zeros(0, dtype=torch.int64, device="cuda"), 2, 1, None,
                                           torch.zeros(1, dtype=torch.float64, device="cuda"), precision, out)
    B.cos_sync_status()
    assert out.shape == (0,)
    M4s = [rand_m4(9950 + c, 1, 2, n)[0] for c, n in enumerate([5, 5, 6, 5])]
    with pytest.raises(B.CosError) as ei:
        run(M4s, 2, 1, None, n_max=5, precision=precision)
    assert ei.value.status == -2


def test_bipartite_deterministic():
    M4s = rand_m4(33, 40, 2, 5)
    a, _ = run(M4s, 2, 1, [[0.1, -0.1], [0.05, 0.02]])
    b, _ = run(M4s, 2, 1, [[0.1, -0.1], [0.05, 0.02]])
    assert np.array_equal(a, b)


def small_hc_model():
    m = I.WORKLOADS["hc_su2_af_n8"].model
    return I.HoneycombModel(6, m.t, m.beta, m.U, (0.1, -0.05), (0.02, 0.0), m.delta, 257)


def test_honeycomb_tables_match_oracle():
    for model in (small_hc_model(), I.WORKLOADS["hc_su2_af_n8"].model):
        tabs = B.honeycomb_tables_for(model)
        got = tabs.table().cpu().numpy()
        ref = HC.hc_model_tables(model)
        assert got.shape == ref.shape
        assert np.max(np.abs(got - ref)) < 1e-13
        inf = tabs.info()
        assert inf.bipartite == 1
        for l in range(model.n_flavors):
            assert list(inf.sigma2[l]) == pytest.approx(list(model.sigma2[l]), rel=1e-15)
        tabs.close()


def test_honeycomb_symmetric_tables_collapse():
    m = I.HoneycombModel(4, 1.0, 3.0, 2.0, (0.1, 0.1), (0.0, 0.0), (0.2, 0.2), 65)
    tabs = B.honeycomb_tables_for(m)
    inf = tabs.info()
    assert inf.symmetric == 1 and inf.n_mat == 1
    tabs.close()


def test_bipartite_gather_and_batch_vs_oracle():
    model = small_hc_model()
    cfgs = I.make_configs(model, 3, 6, 60, 11)
    tabs = B.honeycomb_tables_for(model)
    d = B.configs_to_device(cfgs)
    moff = B.bipartite_matrix_offsets(cfgs.order, 2)
    total = int(moff[-1] + 2 * (2 * int(cfgs.order[-1])) ** 2)
    M4 = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
    B.cos_gather_bipartite(tabs, *d, torch.tensor(moff, device="cuda"), M4)
    out = torch.full((60,), float("nan"), dtype=torch.float64, device="cuda")
    mass = torch.full_like(out, float("nan"))
    B.cos_connected_sum_bipartite_batch(tabs, 6, *d, "fp64", out, mass)
    B.cos_sync_status()
    g = M4.cpu().numpy()
    otabs = HC.hc_model_tables(model)
    s2 = np.array(model.sigma2)
    got, gmass = out.cpu().numpy(), mass.cpu().numpy()
    for c in (0, 17, 59):
        n = int(cfgs.order[c])
        o = int(cfgs.offset[c])
        ref_M4 = HC.hc_gather_one(otabs, cfgs.site[o:o + n], cfgs.tau[o:o + n], model.L, model.beta)
        blk = g[moff[c]:moff[c] + 2 * 4 * n * n].reshape(2, n, 2, n, 2)
        assert np.max(np.abs(blk - ref_M4)) < 1e-13
        ref = O.bip(ref_M4, s2, method="sum_dp", prec="ld")
        rmass = O.bip(ref_M4, s2, method="sum_dp", absmode=True)
        assert abs(got[c] - ref) <= bound(n, rmass) + 1e-13 * rmass, (c, got[c], ref)
        assert gmass[c] == pytest.approx(rmass, rel=1e-10)
    tabs.close()


def test_workload_honeycomb_order8_sampled():
    """SU(2) honeycomb with an antiferromagnetic staggered shift, n = 8, at the benchmark's size
    (2 x 10^4 configurations): sampled configurations against the oracle's sum over the 256
    sublattice assignments."""
    w = I.WORKLOADS["hc_su2_af_n8"]
    nc = w.n_cfg
    cfgs = I.workload_configs(w)
    tabs = B.honeycomb_tables_for(w.model)
    d = B.configs_to_device(cfgs)
    out = torch.full((nc,), float("nan"), dtype=torch.float64, device="cuda")
    B.cos_connected_sum_bipartite_batch(tabs, 8, *d, "fp64", out)
    outm = torch.full_like(out, float("nan"))
    B.cos_connected_sum_bipartite_batch(tabs, 8, *d, "mixed", outm)
    B.cos_sync_status()
    got = out.cpu().numpy()
    gotm = outm.cpu().numpy()
    assert np.all(np.isfinite(got)) and np.all(np.isfinite(gotm))
    otabs = HC.hc_model_tables(w.model)
    s2 = np.array(w.model.sigma2)
    for c in (0, nc // 2, nc - 1):
        o = int(cfgs.offset[c])
        M4 = HC.hc_gather_one(otabs, cfgs.site[o:o + 8], cfgs.tau[o:o + 8], w.model.L, w.model.beta)
        ref = O.bip(M4, s2, method="sum_dp", prec="ld")
        rmass = O.bip(M4, s2, method="sum_dp", absmode=True)
        assert abs(got[c] - ref) <= max(1e-10 * abs(ref), bound(8, rmass)), (c, got[c], ref, rmass)
        assert abs(gotm[c] - ref) <= mixed_bound(8, rmass), (c, gotm[c], ref, rmass)
    tabs.close()


# ------------------------------------------------------------------ gradient (reverse sweep)
# c_bip is quadratic in every single M4 entry (per assignment a vertex-matrix entry is used at
# most twice per cover; the determinant-weight sum is even linear), so central differences of
# the __float128 oracle are exact up to rounding; dc/dsigma2 (dc/dalpha2) from an exact
# polynomial fit; tolerance |err| <= 1e-9 (|ref| + largest reference entry).

def run_bip_grad(M4s, n_mat, wt, s2, gout, det=False, n_max=None):
    order = np.array([m.shape[1] for m in M4s], dtype=np.int32)
    n_max = int(order.max()) if n_max is None else n_max
    moff = B.bipartite_matrix_offsets(order, n_mat)
    d_order = torch.tensor(order, device="cuda")
    d_moff = torch.tensor(moff, device="cuda")
    d_M = torch.tensor(np.concatenate([m.ravel() for m in M4s]), device="cuda")
    nc = len(M4s)
    out = torch.full((nc,), float("nan"), dtype=torch.float64, device="cuda")
    gM = torch.full_like(d_M, float("nan"))
    gs = torch.full((nc, n_mat, 2), float("nan"), dtype=torch.float64, device="cuda")
    g = torch.tensor(gout, dtype=torch.float64, device="cuda")
    if det:
        B.cos_connected_det_bipartite_matrices_grad(n_max, d_order, d_moff, s2, d_M, g, out, gM, gs)
    else:
        B.cos_connected_sum_bipartite_matrices_grad(n_max, d_order, d_moff, n_mat, wt, s2, d_M, g, out, gM, gs)
    B.cos_sync_status()
    gm = gM.cpu().numpy()
    return (out.cpu().numpy(), [gm[moff[c]:moff[c] + m.size].reshape(m.shape) for c, m in enumerate(M4s)],
            gs.cpu().numpy())


def _val(M4, s2, wt, det):
    if det:
        return O.det_clow(M4, s2, prec="q")
    return O.bip(M4, s2, weight=wt, method="dp4", prec="q")


def exact_dM4(M4, s2, wt, det, h=0.25):
    g = np.zeros_like(M4)
    for idx in np.ndindex(*M4.shape):
        Mp = M4.copy(); Mp[idx] += h
        Mm = M4.copy(); Mm[idx] -= h
        g[idx] = (_val(Mp, s2, wt, det) - _val(Mm, s2, wt, det)) / (2 * h)
    return g


def exact_dsig2(M4, s2, wt, det):
    n = M4.shape[1]
    nf = M4.shape[0]
    base = np.zeros((nf, 2)) if s2 is None else np.array(s2, dtype=np.float64)
    out = np.zeros((nf, 2))
    for l in range(nf):
        for s in range(2):
            hs = [0.05 * k for k in range(-n - 1, n + 2)]
            vals = []
            for h in hs:
                t = base.copy(); t[l, s] += h
                vals.append(_val(M4, t, wt, det))
            out[l, s] = np.polyfit(hs, vals, n + 1)[-2]
    return out


def close_to(a, b, rel=1e-9):
    scale = max(np.max(np.abs(b)), 1e-300)
    return np.all(np.abs(a - b) <= rel * (np.abs(b) + scale))


@pytest.mark.parametrize("n,n_mat,wt,shifts,ncfg,det", [
    (1, 2, 1, True, 3, False), (2, 1, 2, False, 5, False), (3, 2, 1, True, 7, False), (4, 2, 1, False, 3, False),
    (3, 1, 3, True, 4, False),   # loop weight 3 with shifts: the non-unit-weight sweep and dsigma
    (1, 2, 1, True, 3, True), (2, 2, 1, False, 5, True), (3, 2, 1, True, 4, True), (4, 2, 1, True, 3, True),
])
def test_bipartite_grad_vs_exact_differences(n, n_mat, wt, shifts, ncfg, det):
    M4s = rand_m4(9000 + 10 * n + n_mat + (100 if det else 0), ncfg, n_mat, n)
    s2 = [[0.08 - 0.05 * l, -0.06 + 0.04 * l] for l in range(n_mat)] if shifts else None
    gout = np.linspace(0.5, 1.5, ncfg)
    out, gM, gs = run_bip_grad(M4s, n_mat, wt, s2, gout, det)
    for c in sorted({0, ncfg - 1}):
        ref = _val(M4s[c], s2, wt, det)
        rmass = (O.det_clow(M4s[c], s2, absmode=True) if det
                 else O.bip(M4s[c], s2, weight=wt, method="sum_dp", absmode=True))
        assert abs(out[c] - ref) <= bound(n, rmass)
        dM = gout[c] * exact_dM4(M4s[c], s2, wt, det)
        assert close_to(gM[c], dM), c
        assert close_to(gs[c], gout[c] * exact_dsig2(M4s[c], s2, wt, det), rel=1e-7), c
        if det:   # dc/dalpha_{b,s} = -sum_j dc/dM4_b[j,s,j,s]
            tr = np.array([[np.trace(dM[b, :, s, :, s]) for s in range(2)] for b in range(2)])
            assert close_to(gs[c], -tr), c


@pytest.mark.parametrize("det", [False, True])
def test_bipartite_grad_orders_7_8_euler(det):
    """Orders 7 and 8: c(t M4, t sigma2) = t^(2n) c gives sum M4 dc/dM4 + sum sigma2 dc/dsigma2 = 2n c;
    the forward value equals the bipartite sweep's bit for bit."""
    orders = [8, 7, 8]
    s2 = [[0.07, -0.03], [0.02, 0.05]]
    M4s = [rand_m4(9500 + c, 1, 2, n)[0] for c, n in enumerate(orders)]
    out, gM, gs = run_bip_grad(M4s, 2, 1, s2, np.ones(len(M4s)), det)
    order = np.array(orders, dtype=np.int32)
    moff = B.bipartite_matrix_offsets(order, 2)
    ref = torch.empty(len(M4s), dtype=torch.float64, device="cuda")
    args = (8, torch.tensor(order, device="cuda"), torch.tensor(moff, device="cuda"))
    d_M = torch.tensor(np.concatenate([m.ravel() for m in M4s]), device="cuda")
    if det:
        B.cos_connected_det_bipartite_matrices(*args, s2, d_M, "fp64", ref)
    else:
        B.cos_connected_sum_bipartite_matrices(*args, 2, 1, s2, d_M, "fp64", ref)
    B.cos_sync_status()
    assert np.array_equal(out, ref.cpu().numpy())
    for c, n in enumerate(orders):
        terms = M4s[c] * gM[c]
        lhs = terms.sum() + float((np.array(s2) * gs[c]).sum())
        scale = np.abs(terms).sum() + float(np.abs(np.array(s2) * gs[c]).sum()) + 2 * n * abs(out[c])
        assert abs(lhs - 2 * n * out[c]) <= 1e-9 * scale, (c, n, lhs, 2 * n * out[c])


@pytest.mark.parametrize("det", [False, True])
def test_bipartite_grad_global_accumulators_bitwise(det):
    """n_max = 9 keeps dc/dM4 in the workspace instead of shared memory: on orders up to 8 the
    gradient is bit for bit that of the shared-memory sweep (n_max = 8)."""
    orders = [8, 5, 8, 7]
    s2 = [[0.05, -0.04], [0.03, 0.06]]
    M4s = [rand_m4(9600 + c, 1, 2, n)[0] for c, n in enumerate(orders)]
    gout = np.linspace(0.7, 1.3, len(M4s))
    a = run_bip_grad(M4s, 2, 1, s2, gout, det, n_max=8)
    b = run_bip_grad(M4s, 2, 1, s2, gout, det, n_max=9)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y)


def test_bipartite_grad_order9():
    """Order 9 (accumulators in the workspace): Euler's relation for both sweeps, the forward
    values equal the bipartite sweeps' bit for bit, and the CoS relation carried to the
    gradient: with two flavors, loop weight 1 and no shifts dc_CoS/dM4 = 2^9 dc_det/dM4."""
    M4s = rand_m4(9650, 2, 2, 9, 0.8)
    order = np.array([9, 9], dtype=np.int32)
    moff = B.bipartite_matrix_offsets(order, 2)
    d_M = torch.tensor(np.concatenate([m.ravel() for m in M4s]), device="cuda")
    args = (9, torch.tensor(order, device="cuda"), torch.tensor(moff, device="cuda"))
    s2 = [[0.06, -0.03], [0.02, 0.04]]
    for det in (False, True):
        out, gM, gs = run_bip_grad(M4s, 2, 1, s2, np.ones(2), det)
        ref = torch.empty(2, dtype=torch.float64, device="cuda")
        if det:
            B.cos_connected_det_bipartite_matrices(*args, s2, d_M, "fp64", ref)
        else:
            B.cos_connected_sum_bipartite_matrices(*args, 2, 1, s2, d_M, "fp64", ref)
        B.cos_sync_status()
        assert np.array_equal(out, ref.cpu().numpy())
        for c in range(2):
            terms = M4s[c] * gM[c]
            lhs = terms.sum() + float((np.array(s2) * gs[c]).sum())
            scale = np.abs(terms).sum() + float(np.abs(np.array(s2) * gs[c]).sum()) + 18 * abs(out[c])
            assert abs(lhs - 18 * out[c]) <= 1e-9 * scale, (det, c, lhs, 18 * out[c])
    _, g_cos, _ = run_bip_grad(M4s, 2, 1, None, np.ones(2), False)
    _, g_det, _ = run_bip_grad(M4s, 2, 1, None, np.ones(2), True)
    for c in range(2):
        scale = np.abs(g_cos[c]).max()
        assert np.max(np.abs(g_cos[c] - 2.0 ** 9 * g_det[c])) <= 1e-9 * scale, c


@pytest.mark.parametrize("det", [False, True])
def test_bipartite_autograd_function(det):
    """torch.autograd through the bipartite sums equals the reverse sweep's gradient, weighted."""
    M4s = rand_m4(9700 + int(det), 4, 2, 4)
    order = np.array([4] * 4, dtype=np.int32)
    moff = B.bipartite_matrix_offsets(order, 2)
    M4 = torch.tensor(np.concatenate([m.ravel() for m in M4s]), device="cuda", requires_grad=True)
    s2v = [[0.06, -0.02], [0.03, 0.05]]
    s2 = torch.tensor(s2v, dtype=torch.float64, requires_grad=True)
    w = torch.linspace(0.5, 1.5, 4, dtype=torch.float64, device="cuda")
    d_order, d_moff = torch.tensor(order, device="cuda"), torch.tensor(moff, device="cuda")
    if det:
        c = AG.connected_det_bipartite(M4, s2, d_order, d_moff, 4)
    else:
        c = AG.connected_sum_bipartite(M4, s2, d_order, d_moff, 4, 2, 1)
    (c * w).sum().backward()
    out, gM, gs = run_bip_grad(M4s, 2, 1, s2v, w.cpu().numpy(), det)
    assert np.array_equal(c.detach().cpu().numpy(), out)
    assert np.array_equal(M4.grad.cpu().numpy(), np.concatenate([g.ravel() for g in gM]))
    assert np.allclose(s2.grad.numpy(), gs.sum(0), rtol=1e-14, atol=0)


@pytest.mark.parametrize("sym", [False, True])
def test_bipartite_grad_from_coordinates(sym):
    """dLoss/dM4 from vertex coordinates is the matrices entry's on the blocks
    cos_gather_bipartite writes (bitwise); dLoss/dmu and dLoss/dalpha match central differences
    of the oracle pipeline (honeycomb tables, gather, the sum over sublattice assignments)
    rebuilt at mu +- h and alpha +- h.  Collapsed tables move every flavor together and split
    the derivative evenly."""
    base = I.WORKLOADS["hc_su2_af_n8"].model
    mu = [0.1, 0.1] if sym else [-0.15, 0.2]
    alpha = [0.05, 0.05] if sym else [0.1, -0.05]
    delta = (0.25, 0.25) if sym else base.delta
    mk = lambda m, a: I.HoneycombModel(base.L, base.t, base.beta, base.U, tuple(m), tuple(a), delta, base.n_tau)
    model = mk(mu, alpha)
    nc = 24
    cfgs = I.make_configs(model, 3, 5, nc, 31)
    tabs = B.honeycomb_tables_for(model)
    info = tabs.info()
    n_mat = info.n_mat
    assert n_mat == (1 if sym else 2)
    d = B.configs_to_device(cfgs)
    order = cfgs.order.astype(np.int32)
    total = int(n_mat * 4 * (order.astype(np.int64) ** 2).sum())
    gmoff = torch.tensor(B.bipartite_matrix_offsets(order, n_mat), device="cuda")
    gout = np.linspace(0.5, 1.5, nc)
    g = torch.tensor(gout, device="cuda")
    nan = float("nan")
    out = torch.full((nc,), nan, dtype=torch.float64, device="cuda")
    gM = torch.full((total,), nan, dtype=torch.float64, device="cuda")
    gmu = torch.full((nc, 2), nan, dtype=torch.float64, device="cuda")
    ga = torch.full_like(gmu, nan)
    B.cos_connected_sum_bipartite_grad(tabs, 5, *d, g, out, gM, gmoff, gmu, ga)
    M4 = torch.empty(total, dtype=torch.float64, device="cuda")
    B.cos_gather_bipartite(tabs, *d, gmoff, M4)
    s2 = [[info.sigma2[l][s] for s in range(2)] for l in range(n_mat)]
    wt = info.n_flavors if info.symmetric else 1
    out2 = torch.full_like(out, nan)
    gM2 = torch.full_like(gM, nan)
    B.cos_connected_sum_bipartite_matrices_grad(5, d[0], gmoff, n_mat, wt, s2, M4, g, out2, gM2, None)
    B.cos_sync_status()
    tabs.close()
    assert np.array_equal(out.cpu().numpy(), out2.cpu().numpy())
    assert np.array_equal(gM.cpu().numpy(), gM2.cpu().numpy())
    gmu, ga = gmu.cpu().numpy(), ga.cpu().numpy()

    picks = (0, nc // 2, nc - 1)

    def oracle_c(m2, a2):
        m = mk(m2, a2)
        t = HC.hc_model_tables(m)
        vals = []
        for c in picks:
            o, n = int(cfgs.offset[c]), int(cfgs.order[c])
            G4 = HC.hc_gather_one(t, cfgs.site[o:o + n], cfgs.tau[o:o + n], m.L, m.beta)
            vals.append(O.bip(G4, np.array(m.sigma2), method="sum_dp", prec="ld"))
        return np.array(vals)

    h = 1e-6
    for which, base_v, got in (("mu", mu, gmu), ("alpha", alpha, ga)):
        for l in range(2):
            if sym:
                p = [x + h for x in base_v]
                q = [x - h for x in base_v]
            else:
                p = list(base_v); p[l] += h
                q = list(base_v); q[l] -= h
            args_p = (p, alpha) if which == "mu" else (mu, p)
            args_q = (q, alpha) if which == "mu" else (mu, q)
            fd = (oracle_c(*args_p) - oracle_c(*args_q)) / (2 * h) / (2 if sym else 1)
            for k, c in enumerate(picks):
                want = gout[c] * fd[k]
                assert got[c, l] == pytest.approx(want, rel=2e-5, abs=1e-7 * max(1.0, abs(want))), \
                    (which, l, c, got[c, l], want)


def test_bipartite_model_autograd():
    """connected_sum_bipartite_model: the forward equals cos_connected_sum_bipartite_batch bit for
    bit, and mu.grad / alpha.grad are cos_connected_sum_bipartite_grad's per-configuration
    gradients summed with the weights."""
    base = I.WORKLOADS["hc_su2_af_n8"].model
    mu, alpha = [-0.1, 0.15], [0.05, -0.02]
    model = I.HoneycombModel(base.L, base.t, base.beta, base.U, tuple(mu), tuple(alpha), base.delta, base.n_tau)
    nc = 48
    cfgs = I.make_configs(model, 3, 6, nc, 41)
    d = B.configs_to_device(cfgs)
    mu_t = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
    al_t = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    c = AG.connected_sum_bipartite_model(mu_t, al_t, model, d, 6)
    w = torch.linspace(-1.0, 2.0, nc, dtype=torch.float64, device="cuda")
    (c * w).sum().backward()
    tabs = B.honeycomb_tables_for(model)
    ref = torch.empty(nc, dtype=torch.float64, device="cuda")
    B.cos_connected_sum_bipartite_batch(tabs, 6, *d, "fp64", ref)
    gmu = torch.empty(nc, 2, dtype=torch.float64, device="cuda")
    gal = torch.empty_like(gmu)
    B.cos_connected_sum_bipartite_grad(tabs, 6, *d, w, gmu=gmu, galpha=gal)
    B.cos_sync_status()
    tabs.close()
    assert np.array_equal(c.detach().cpu().numpy(), ref.cpu().numpy())
    assert np.allclose(mu_t.grad.numpy(), gmu.sum(0).cpu().numpy(), rtol=1e-14, atol=0)
    assert np.allclose(al_t.grad.numpy(), gal.sum(0).cpu().numpy(), rtol=1e-14, atol=0)


@pytest.mark.parametrize("det", [False, True])
def test_bipartite_grad_checkpointed_bitwise_and_exact(monkeypatch, det):
    """The bipartite reverse sweep with the least-storage checkpoint plan forced (segments re-run
    from their checkpoints, each adjoint in place of its forward state): bitwise the gradient
    with every layer kept, at orders 4-7 in one uneven launch, and exact differences at order 4."""
    orders = [6, 4, 7, 5, 7]
    M4s = [rand_m4(9500 + 7 * c + (50 if det else 0), 1, 2, n)[0] for c, n in enumerate(orders)]
    s2 = [[0.07, -0.04], [0.03, 0.05]]
    gout = np.array([1.0, 0.5, -1.5, 2.0, 0.75])
    monkeypatch.setenv("COS_GRAD_CHECKPOINT", "0")
    a = run_bip_grad(M4s, 2, 1, s2, gout, det)
    monkeypatch.setenv("COS_GRAD_CHECKPOINT", "1")
    b = run_bip_grad(M4s, 2, 1, s2, gout, det)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
    assert all(np.array_equal(x, y) for x, y in zip(a[1], b[1]))
    assert close_to(b[1][1], gout[1] * exact_dM4(M4s[1], s2, 1, det))
