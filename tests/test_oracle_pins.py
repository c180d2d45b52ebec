"""Pins of the CPU oracle to what the paper and the mathematics fix.

Each test ties an oracle function to something other than itself: a printed
example, a closed form, a library routine, an invariant or brute force.
P-numbers follow the pin list of the design notes (P0 .. P9).
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from oracle import propagators as P
from paper_2507_12349_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(20250716)


def rnd(*shape):
    return RNG.uniform(-1.0, 1.0, size=shape)


# ------------------------------------------------------------------ golden fixtures

def test_splitmix64_published_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_vectors.txt")) if l[0] != "#"]
    for state, want in rows:
        got = I.splitmix64(np.array([int(state, 16)], dtype=np.uint64))[0]
        assert int(got) == int(want, 16)


def test_mv_cover_sign_example():
    """Results A: cover (1)(2)(3,4) of a 4x4 matrix has sign (-1)^(n-k)."""
    lines = [l.split() for l in open(os.path.join(GOLDEN, "mv_cover_sign.txt")) if l[0] != "#"]
    A = np.zeros((4, 4))
    prod = 1.0
    for i, j, v in lines[:4]:
        A[int(i) - 1, int(j) - 1] = float(v)
        prod *= float(v)
    n, k, sign = (int(x) for x in lines[4])
    assert sign == (-1) ** (n - k)
    # 4 points = 2 vertices; no connectivity filter, one flavor, no shifts
    assert O.brute(A[None], None, connected=False) == pytest.approx(sign * prod, rel=1e-15)
    assert O.brute_py(A[None], None, connected=False) == pytest.approx(sign * prod, rel=1e-15)
    assert O.point_dp(A, connected=False) == pytest.approx(sign * prod, rel=1e-15)


# ------------------------------------------------------------------ P0: determinant

@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_p0_all_covers_one_flavor_is_det(n):
    """Sum over all covers with -1 per loop and one flavor = det(A) (LU)."""
    A = rnd(2 * n, 2 * n)
    ref = np.linalg.det(A)
    assert O.brute(A[None], None, connected=False) == pytest.approx(ref, rel=1e-12, abs=1e-13)
    assert O.brute(A[None], None, connected=False, prec="q") == pytest.approx(ref, rel=1e-12, abs=1e-13)
    assert O.point_dp(A, connected=False) == pytest.approx(ref, rel=1e-12, abs=1e-13)
    if n <= 2:
        assert O.brute_py(A[None], None, connected=False) == pytest.approx(ref, rel=1e-12, abs=1e-13)


# ------------------------------------------------------------------ P1: tiers agree

CASES = [  # (n, nf, shifts)
    (1, 1, False), (1, 3, True), (2, 2, False), (2, 3, True), (3, 1, True), (3, 2, True),
    (3, 4, False), (4, 2, True), (4, 3, False),
]


@pytest.mark.parametrize("n,nf,shifts", CASES)
def test_p1_brute_closed_dp_agree(n, nf, shifts):
    M = rnd(nf, n, n)
    sig = rnd(nf) if shifts else None
    ref = O.brute(O.tiled(M), sig, prec="q")
    mass = O.dp(M, sig, absmode=True)
    tol = 1e-13 * mass
    assert O.brute(O.tiled(M), sig) == pytest.approx(ref, abs=tol)
    assert O.closed(M, sig, prec="q") == pytest.approx(ref, abs=tol)
    assert O.closed(M, sig) == pytest.approx(ref, abs=tol)
    assert O.dp(M, sig, prec="q") == pytest.approx(ref, abs=tol)
    assert O.dp(M, sig, prec="ld") == pytest.approx(ref, abs=tol)
    assert O.dp(M, sig) == pytest.approx(ref, abs=tol)
    if n <= 2 or (n == 3 and nf <= 2):
        assert O.brute_py(O.tiled(M), sig) == pytest.approx(ref, abs=tol)


@pytest.mark.slow
def test_p1_brute_n5_shifts():
    M = rnd(3, 5, 5)
    sig = rnd(3)
    ref = O.brute(O.tiled(M), sig)
    mass = O.dp(M, sig, absmode=True)
    assert O.dp(M, sig, prec="q") == pytest.approx(ref, abs=1e-13 * mass)
    assert O.closed(M, sig, prec="q") == pytest.approx(ref, abs=1e-13 * mass)


@pytest.mark.parametrize("n,wt", [(2, 1), (2, 3), (3, 2), (3, 6), (4, 4)])
def test_p1_unmerged_point_dp_equals_merged(n, wt):
    """Alg. 2 on points (visited set R) equals the merged ternary-mask DP."""
    M = rnd(1, n, n)
    ref = O.dp(M, None, weight=wt, prec="q")
    assert O.point_dp(O.tiled(M)[0], weight=wt) == pytest.approx(ref, abs=1e-12 * O.dp(M, None, wt, absmode=True))


def test_p1_symmetric_weight_equals_flavor_copies():
    """One matrix with loop weight N equals N identical flavors (sum over flavors)."""
    n, N = 5, 4
    M = rnd(1, n, n)
    sig = 0.3
    a = O.dp(M, [sig], weight=N, prec="q")
    b = O.dp(np.repeat(M, N, axis=0), [sig] * N, prec="q")
    assert a == pytest.approx(b, rel=1e-13)


# ------------------------------------------------------------------ P2: SU(2) identity

def cdet_su2(M):
    """CDet with a(S) = det(M[S])^2 and the subset subtraction (Methods A)."""
    n = M.shape[0]
    a = {}
    for S in range(1 << n):
        idx = [i for i in range(n) if S >> i & 1]
        a[S] = np.linalg.det(M[np.ix_(idx, idx)]) ** 2 if idx else 1.0
    c = {}
    for T in range(1, 1 << n, 2):          # subsets containing vertex 0
        acc = a[T]
        for Tp in range(1, T, 2):          # proper subsets of T containing vertex 0
            if Tp & ~T:
                continue
            acc -= c[Tp] * a[T & ~Tp]
        c[T] = acc
    return c[(1 << n) - 1]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 8])
def test_p2_su2_is_2n_cdet(n):
    M = rnd(n, n)
    ref = 2 ** n * cdet_su2(M)
    mass = O.dp(M[None], None, weight=2, absmode=True)
    assert O.dp(M[None], None, weight=2, prec="q") == pytest.approx(ref, abs=1e-12 * mass)
    assert O.closed(np.stack([M, M]), None, prec="q") == pytest.approx(ref, abs=1e-12 * mass)
    if n <= 3:
        assert O.brute(O.tiled(np.stack([M, M]))) == pytest.approx(ref, abs=1e-12 * mass)


# ------------------------------------------------------------------ P3: Pauli zero

@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_p3_one_flavor_vanishes(n):
    M = rnd(1, n, n)
    mass = O.dp(M, None, absmode=True)
    assert abs(O.dp(M, None, prec="q")) < 1e-14 * mass
    assert abs(O.closed(M, None, prec="q")) < 1e-14 * mass
    if n <= 4:
        assert abs(O.brute(O.tiled(M))) < 1e-13 * mass


# ------------------------------------------------------------------ P4: subset exponential

def set_partitions(items):
    if not items:
        yield []
        return
    first, rest = items[0], items[1:]
    for part in set_partitions(rest):
        for k in range(len(part)):
            yield part[:k] + [[first] + part[k]] + part[k + 1:]
        yield [[first]] + part


@pytest.mark.parametrize("n,nf,shifts", [(3, 2, True), (4, 2, False), (4, 3, True)])
def test_p4_all_covers_is_exponential_of_connected(n, nf, shifts):
    M = rnd(nf, n, n)
    sig = rnd(nf) if shifts else None
    a_all = O.brute(O.tiled(M), sig, connected=False, prec="q")
    total = 0.0
    for part in set_partitions(list(range(n))):
        w = 1.0
        for block in part:
            sub = M[:, block][:, :, block]
            w *= O.dp(sub, sig, prec="q")
        total += w
    assert total == pytest.approx(a_all, rel=1e-12)
    # and the closed form's a(S) for every subset against brute force
    _, a_sub, _ = O.closed(M, sig, prec="q", subsets=True)
    for S in range(1, 1 << n):
        idx = [i for i in range(n) if S >> i & 1]
        ref = O.brute(O.tiled(M[:, idx][:, :, idx]), sig, connected=False, prec="q")
        assert a_sub[S] == pytest.approx(ref, rel=1e-11, abs=1e-13)


# ------------------------------------------------------------------ P5: symmetric limit

@pytest.mark.parametrize("n,N", [(1, 2), (2, 2), (2, 3), (3, 3), (4, 2)])
def test_p5_symmetric_limit_is_diagonal_shift(n, N):
    """Broken run with equal flavors and sigma equals CoS (weight N per loop) on
    the point matrix with diagonal A_pp + sigma/N (Methods A, equal-time
    shift alpha/(N_f U) for CoS); at n = 1 they differ by sigma^2 (the
    double-shift term excluded by at most one shift per vertex)."""
    M = rnd(1, n, n)
    s = 0.37
    broken = O.dp(np.repeat(M, N, axis=0), [s] * N, prec="q")
    A = O.tiled(M)[0] + np.eye(2 * n) * s / N
    cos_diag = O.brute(np.repeat(A[None], N, axis=0), None, prec="q")
    extra = s * s if n == 1 else 0.0
    assert broken + extra == pytest.approx(cos_diag, rel=1e-12)


# ------------------------------------------------------------------ P6: n = 1

def test_p6_order_one_closed_form():
    g = rnd(4)
    sig = rnd(4)
    M = g.reshape(4, 1, 1)
    ref = sum(g[a] * g[b] for a in range(4) for b in range(4) if a != b) + 2 * float(np.dot(sig, g))
    for f in (lambda: O.dp(M, sig), lambda: O.closed(M, sig), lambda: O.brute(O.tiled(M), sig)):
        assert f() == pytest.approx(ref, rel=1e-14)
    # symmetric N_f: N(N-1) g^2
    assert O.dp(M[:1], None, weight=6) == pytest.approx(30 * g[0] ** 2, rel=1e-14)


# ------------------------------------------------------------------ P7: invariances

@pytest.mark.parametrize("n,nf,shifts", [(6, 3, True), (7, 2, False), (8, 1, False)])
def test_p7_invariances(n, nf, shifts):
    M = rnd(nf, n, n)
    sig = rnd(nf) if shifts else None
    wt = 4 if nf == 1 else 1
    base = O.dp(M, sig, weight=wt, prec="ld")
    tol = 1e-12 * O.dp(M, sig, weight=wt, absmode=True)
    # transpose
    assert O.dp(M.transpose(0, 2, 1), sig, weight=wt, prec="ld") == pytest.approx(base, abs=tol)
    # vertex relabeling (tests the head rule's canonical choice)
    perm = RNG.permutation(n)
    assert O.dp(M[:, perm][:, :, perm], sig, weight=wt, prec="ld") == pytest.approx(base, abs=tol)
    # flavor relabeling
    fp = RNG.permutation(nf)
    assert O.dp(M[fp], None if sig is None else sig[fp], weight=wt, prec="ld") == pytest.approx(base, abs=tol)
    # diagonal similarity shared by all flavors
    d = RNG.uniform(0.5, 2.0, size=n)
    Ms = M * d[None, :, None] / d[None, None, :]
    assert O.dp(Ms, sig, weight=wt, prec="ld") == pytest.approx(base, abs=tol * 4)
    # homogeneity of degree 2n in (M, sigma)
    s = 0.7
    got = O.dp(s * M, None if sig is None else s * sig, weight=wt, prec="ld")
    assert got == pytest.approx(s ** (2 * n) * base, abs=tol * s ** (2 * n))
    # the closed form agrees at this size
    if n <= 7:
        assert O.closed(np.repeat(M, wt, axis=0) if wt > 1 else M,
                        None if sig is None else (np.repeat(sig, wt) if wt > 1 else sig),
                        prec="ld") == pytest.approx(base, abs=tol)


def test_mass_bounds_value():
    for n in (3, 5, 6):
        M = rnd(3, n, n)
        sig = rnd(3)
        assert O.dp(M, sig, absmode=True) >= abs(O.dp(M, sig))
        assert O.dp(np.abs(M), np.abs(sig), absmode=True) == pytest.approx(O.dp(M, sig, absmode=True))


# ------------------------------------------------------------------ P8: gradient

def test_p8_connected_sum_is_quadratic_in_each_entry():
    """Each vertex has two points, so a cover uses M^l[a][b] at most twice:
    c is a quadratic polynomial in every single entry, and its third
    difference vanishes (central differences are then exact)."""
    n, nf = 4, 3
    M = rnd(nf, n, n)
    sig = rnd(nf)
    for (l, a, b) in [(0, 0, 0), (1, 2, 3), (2, 3, 1)]:
        vals = []
        for k in range(4):
            Mk = M.copy()
            Mk[l, a, b] += 0.5 * k
            hi, lo = O.dp(Mk, sig, prec="q", pair=True)
            vals.append(Fraction(hi) + Fraction(lo))      # exact sum of the pair
        third = vals[3] - 3 * vals[2] + 3 * vals[1] - vals[0]
        assert abs(float(third)) < 1e-25 * max(abs(float(v)) for v in vals)


def fd_grad_M(M, sig, h=0.25):
    """Central differences of the __float128 DP: exact for a quadratic."""
    g = np.zeros_like(M)
    for idx in np.ndindex(*M.shape):
        Mp = M.copy(); Mp[idx] += h
        Mm = M.copy(); Mm[idx] -= h
        g[idx] = (O.dp(Mp, sig, prec="q") - O.dp(Mm, sig, prec="q")) / (2 * h)
    return g


@pytest.mark.parametrize("n,nf,shifts", [(1, 3, True), (2, 2, True), (3, 2, False), (3, 2, True)])
def test_p8_autograd_of_dense_brute_matches_exact_differences(n, nf, shifts):
    torch = pytest.importorskip("torch")
    M = rnd(nf, n, n)
    sig = rnd(nf) if shifts else None
    Mt = torch.tensor(M, dtype=torch.float64, requires_grad=True)
    st = torch.tensor(sig, dtype=torch.float64, requires_grad=True) if shifts else None
    c = O.torch_brute(Mt, st)
    assert float(c) == pytest.approx(O.dp(M, sig, prec="q"), rel=1e-12, abs=1e-14)
    c.backward()
    assert np.allclose(Mt.grad.numpy(), fd_grad_M(M, sig), rtol=1e-11, atol=1e-13)
    if shifts:
        # sigma enters with degree up to n: Richardson-free check by a polynomial fit
        for l in range(nf):
            hs = [0.05 * k for k in range(-n - 1, n + 2)]
            vals = []
            for h in hs:
                s2 = sig.copy(); s2[l] += h
                vals.append(O.dp(M, s2, prec="q"))
            coef = np.polyfit(hs, vals, n + 1)
            assert st.grad[l].item() == pytest.approx(coef[-2], rel=1e-8, abs=1e-10)


# ------------------------------------------------------------------ P9: propagator tables

def test_p9_half_filling_and_jump():
    L, beta, n_tau = 8, 2.0, 65
    tab = P.table(L, 1.0, beta, 0.0, 0.0, n_tau)
    g0m = -tab[:, -1]                        # G(r, 0^-) = -G(r, beta^-)
    assert g0m[0] == pytest.approx(0.5, abs=1e-14)     # particle-hole symmetric square lattice
    # jump G(0^+) - G(0^-) = -delta_{r,0} (anticommutator)
    jump = tab[:, 0] - g0m
    want = np.zeros(L * L); want[0] = -1.0
    assert np.allclose(jump, want, atol=1e-14)


def test_p9_momentum_zero_sum_and_antiperiodic():
    L, beta, n_tau, mu, alpha = 6, 3.0, 33, 0.4, -0.1
    tab = P.table(L, 1.0, beta, mu, alpha, n_tau)
    xi0 = -4.0 - mu + alpha
    nf0 = 1.0 / (math.exp(beta * xi0) + 1.0)
    assert (-tab[:, -1]).sum() == pytest.approx(nf0, rel=1e-13)   # sum_r G(r,0^-) = n_F(xi_{k=0})
    # interpolation: at dt = 0 the value is G(0^-); at dt -> dt - beta the sign flips
    r = 7
    assert P.interp(tab, r, 0.0, beta) == pytest.approx(-tab[r, -1], rel=1e-15)
    dt = 0.7 * beta / (n_tau - 1) * 5
    assert P.interp(tab, r, dt - beta, beta) == pytest.approx(-P.interp(tab, r, dt, beta), rel=1e-15)


def test_p9_single_site_closed_form():
    """L = 1: one momentum, xi = -4t - mu + alpha, G(tau) = -exp(-xi tau)(1 - n_F)."""
    beta, n_tau, mu, alpha = 5.0, 11, 0.3, 0.2
    xi = -4.0 - mu + alpha
    tab = P.table(1, 1.0, beta, mu, alpha, n_tau)
    tg = P.tau_grid(beta, n_tau)
    want = -np.exp(-xi * tg) * (1.0 - 1.0 / (np.exp(beta * xi) + 1.0))
    assert np.allclose(tab[0], want, rtol=1e-13)


def test_p9_dmu_table_is_derivative():
    L, beta, n_tau, mu = 4, 4.0, 17, -0.2
    h = 1e-5
    d = P.dtable_dmu(L, 1.0, beta, mu, 0.0, n_tau)
    fd = (P.table(L, 1.0, beta, mu + h, 0.0, n_tau) - P.table(L, 1.0, beta, mu - h, 0.0, n_tau)) / (2 * h)
    assert np.allclose(d, fd, rtol=1e-7, atol=1e-10)


def test_gather_uses_displacement_and_equal_time_convention():
    model = I.Model(4, 1.0, 2.0, 1.0, (0.1, -0.2), (0.0, 0.0), 9)
    tabs = P.model_tables(model)
    sites = [0, 5, 15]
    taus = [0.3, 0.3, 1.9]
    M = P.gather_one(tabs, sites, taus, 4, 2.0)
    # diagonal and equal times are G(r, 0^-)
    for l in range(2):
        assert M[l, 0, 0] == pytest.approx(-tabs[l, 0, -1])
        assert M[l, 0, 1] == pytest.approx(-tabs[l, P.displacement(0, 5, 4), -1])
    # r_0 - r_2: (0,0) - (3,3) = (1,1) mod 4 -> site 5; dt = -1.6 -> -G(0.4)
    assert P.displacement(0, 15, 4) == 5
    assert M[0, 0, 2] == pytest.approx(-P.interp(tabs[0], 5, 0.4, 2.0) * 1.0)
    assert M[0, 2, 0] == pytest.approx(P.interp(tabs[0], P.displacement(15, 0, 4), 1.6, 2.0))


# ------------------------------------------------------------------ the batch driver

@pytest.mark.parametrize("prec", ["d", "ld"])
@pytest.mark.parametrize("n,nf,shifts,weight", [(3, 1, False, 3), (5, 3, True, 1), (6, 4, False, 1),
                                                (7, 1, True, 6), (4, 2, True, 2)])
def test_dp_batch_equals_dp_per_configuration(prec, n, nf, shifts, weight):
    """The OpenMP batch driver (which feeds the timed CPU baseline and every accuracy figure of
    the benchmark) returns, configuration by configuration, exactly the (hi, lo) pair of the
    pinned single-configuration DP: different matrices per configuration of one order, shift
    weights on and off, loop weights above 1, the absolute-mass mode, one thread and all
    threads.  A stride, offset or sigma-handling slip in the driver changes some bits."""
    rng = np.random.default_rng(1000 * n + 10 * nf + weight)
    n_cfg = 37                                       # not a multiple of any thread count
    Ms = rng.uniform(-0.9, 0.9, size=(n_cfg, nf, n, n))
    sig = list(rng.uniform(-0.3, 0.3, size=nf)) if shifts else None
    for absmode in (False, True):
        want = [O.dp(Ms[c], sig, weight=weight, absmode=absmode, prec=prec, pair=True) for c in range(n_cfg)]
        for threads in (1, 0):
            hi, lo, used = O.dp_batch(Ms, sig, weight, absmode=absmode, prec=prec, nthreads=threads)
            assert used >= 1 and (threads != 1 or used == 1)
            assert [(float(h), float(l)) for h, l in zip(hi, lo)] == want
    # each configuration's own matrices: permuting the batch permutes the results
    perm = rng.permutation(n_cfg)
    hi, lo, _ = O.dp_batch(Ms, sig, weight, prec=prec)
    hp, lp, _ = O.dp_batch(Ms[perm], sig, weight, prec=prec)
    assert np.array_equal(hp, hi[perm]) and np.array_equal(lp, lo[perm])


def test_dp_batch_rejects_unsupported_order():
    with pytest.raises(ValueError):
        O.dp_batch(np.zeros((2, 1, 13, 13)))
