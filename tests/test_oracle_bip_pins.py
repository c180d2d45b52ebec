"""Pins of the bipartite (two-sublattice) oracle and the honeycomb propagators.

Each check compares the oracle with something other than itself:
  * the three single-assignment routes (merged DP, determinants + subset subtraction, brute
    force over decorated covers) summed over all sublattice assignments, and the
    sublattice-resolved merged DP of Alg. 1-2, must agree (independent algorithms);
  * per-vertex shift weights: DP vs brute force vs closed form;
  * equal sublattice blocks: every assignment gives the same matrices, so the sum is
    2^n times the plain connected sum;
  * SU(2) symmetric without shifts: every assignment's CoS value is 2^n times its CDet
    (connected determinant from LU determinants, Methods A recursion) -- pin P2 per
    assignment, summed;
  * n = 1 closed form per sublattice;
  * the honeycomb tables against a 40-digit matrix exponential (L = 1), the equal-time jump,
    half filling, the sum rule and the real-space symmetry G_ss'(R) = G_s's(-R).
"""
import itertools

import numpy as np
import pytest

import oracle as O
from oracle import honeycomb as HC
from oracle.propagators import fermi
from paper_2507_12349_b300 import inputs as I


def rand_m4(seed, nf, n, scale=0.9):
    M = I.random_matrices(seed, 1, nf, 2 * n, scale)[0]          # [nf][2n][2n], index i*2 + s
    return np.ascontiguousarray(M.reshape(nf, n, 2, n, 2))


def rand_sig2(seed, nf):
    u = I.random_matrices(seed + 999, 1, 1, 2 * nf, 0.25)[0, 0, 0]
    return u[: 2 * nf].reshape(nf, 2)


@pytest.mark.parametrize("n,nf", [(1, 1), (1, 3), (2, 2), (3, 1), (3, 2), (4, 2), (4, 3)])
def test_bip_routes_agree(n, nf):
    M4 = rand_m4(10 * n + nf, nf, n)
    s2 = rand_sig2(n + nf, nf)
    ref = O.bip(M4, s2, method="sum_dp", prec="q")
    scale = O.bip(M4, s2, method="sum_dp", absmode=True)
    assert O.bip(M4, s2, method="sum_closed", prec="q") == pytest.approx(ref, abs=1e-13 * scale)
    assert O.bip(M4, s2, method="dp4", prec="q") == pytest.approx(ref, abs=1e-13 * scale)
    if n <= 3:
        assert O.bip(M4, s2, method="sum_brute", prec="ld") == pytest.approx(ref, abs=1e-12 * scale)
    assert O.bip(M4, s2, method="dp4", absmode=True) == pytest.approx(scale, rel=1e-12)


@pytest.mark.parametrize("n,nf", [(5, 2), (6, 1)])
def test_bip_dp4_matches_assignment_sum_larger(n, nf):
    M4 = rand_m4(70 + n, nf, n)
    s2 = rand_sig2(3, nf)
    ref = O.bip(M4, s2, method="sum_dp", prec="ld")
    scale = O.bip(M4, s2, method="sum_dp", absmode=True)
    assert O.bip(M4, s2, method="dp4", prec="ld") == pytest.approx(ref, abs=1e-13 * scale)


def test_per_vertex_shifts_dp_closed_brute():
    for n, nf in [(2, 2), (3, 2), (4, 1)]:
        M = I.random_matrices(40 + n, 1, nf, n, 0.9)[0]
        sv = I.random_matrices(41 + n, 1, 1, nf * n, 0.3)[0, 0, 0][: nf * n].reshape(nf, n)
        ref = O.brute(O.tiled(M), sv)
        scale = O.dp(M, sv, absmode=True)
        assert O.dp(M, sv, prec="ld") == pytest.approx(ref, abs=1e-12 * scale)
        assert O.closed(M, sv, prec="ld") == pytest.approx(ref, abs=1e-12 * scale)
        # a per-vertex array that is constant per flavor is the per-flavor case
        const = np.tile(sv[:, :1], (1, n))
        assert O.dp(M, const, prec="ld") == pytest.approx(O.dp(M, list(sv[:, 0]), prec="ld"), rel=1e-15)


@pytest.mark.parametrize("n,nf", [(3, 2), (5, 1), (6, 2)])
def test_equal_blocks_give_two_to_the_n(n, nf):
    M = I.random_matrices(90 + n, 1, nf, n, 0.9)[0]
    M4 = np.ascontiguousarray(np.broadcast_to(M[:, :, None, :, None], (nf, n, 2, n, 2)))
    sig = rand_sig2(n, nf)[:, 0]
    s2 = np.stack([sig, sig], axis=1)
    scale = O.dp(M, list(sig), absmode=True) * 2 ** n
    ref = 2 ** n * O.dp(M, list(sig), prec="ld")
    assert O.bip(M4, s2, method="dp4", prec="ld") == pytest.approx(ref, abs=1e-13 * scale)


def cdet(M: np.ndarray) -> float:
    """Connected determinant of the SU(2) symmetric weight det(M[S])^2 (Methods A recursion)."""
    n = M.shape[0]
    a = np.zeros(1 << n)
    for S in range(1 << n):
        idx = [i for i in range(n) if S >> i & 1]
        a[S] = np.linalg.det(M[np.ix_(idx, idx)]) ** 2 if idx else 1.0
    c = np.zeros(1 << n)
    for S in range(1, 1 << n):
        low = S & -S
        rest = S ^ low
        acc = a[S]
        R = rest
        while True:
            T = low | R
            if T != S:
                acc -= c[T] * a[S ^ T]
            if R == 0:
                break
            R = (R - 1) & rest
        c[S] = acc
    return c[(1 << n) - 1]


@pytest.mark.parametrize("n", [2, 4, 6])
def test_su2_symmetric_bipartite_is_sum_of_cdet(n):
    M4 = rand_m4(300 + n, 1, n)
    ref = 0.0
    for s in itertools.product(range(2), repeat=n):
        Ms, _ = O.bip_assignment(M4, None, s)
        ref += 2 ** n * cdet(Ms[0])
    got = O.bip(M4, None, weight=2, method="dp4", prec="ld")
    scale = O.bip(M4, None, weight=2, method="dp4", absmode=True)
    assert got == pytest.approx(ref, abs=1e-11 * scale)


def test_n1_closed_form():
    nf = 3
    M4 = rand_m4(5, nf, 1)
    s2 = rand_sig2(5, nf)
    ref = 0.0
    for s in range(2):
        g = M4[:, 0, s, 0, s]
        ref += sum(g[a] * g[b] for a in range(nf) for b in range(nf) if a != b) + 2 * np.dot(s2[:, s], g)
    assert O.bip(M4, s2, method="dp4", prec="ld") == pytest.approx(ref, rel=1e-13)


def test_sublattice_relabeling():
    n, nf = 4, 2
    M4 = rand_m4(12, nf, n)
    s2 = rand_sig2(12, nf)
    M4f = np.ascontiguousarray(M4[:, :, ::-1, :, ::-1])
    s2f = np.ascontiguousarray(s2[:, ::-1])
    a = O.bip(M4, s2, method="dp4", prec="ld")
    b = O.bip(M4f, s2f, method="dp4", prec="ld")
    assert a == pytest.approx(b, abs=1e-13 * O.bip(M4, s2, method="dp4", absmode=True))


# ------------------------------------------------------------------ honeycomb propagators

def test_honeycomb_L1_matches_matrix_exponential():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    beta, mu, alpha, delta = 4.0, 0.2, 0.05, 0.3
    tab = HC.hc_table(1, 1.0, beta, mu, alpha, delta, 9)
    Hk = HC.hc_bloch(1, 1.0, mu, alpha, delta)[0].real
    Hm = mp.matrix(Hk.tolist())
    Id = mp.eye(2)
    nF = mp.inverse(mp.expm(beta * Hm) + Id)
    for m in range(9):
        ref = -(mp.expm(-Hm * (m * beta / 8)) * (Id - nF))
        for s in range(2):
            for t in range(2):
                assert tab[s, t, 0, m] == pytest.approx(float(ref[s, t]), abs=2e-15)


def test_honeycomb_jump_half_filling_symmetry_and_sum_rule():
    L, beta = 6, 4.0
    tab = HC.hc_table(L, 1.0, beta, 0.0, 0.0, 0.0, 129)
    jump = tab[..., 0] + tab[..., -1]            # G(0^+) - G(0^-), G(0^-) = -G(beta^-)
    assert np.allclose(jump[:, :, 0], -np.eye(2), atol=1e-14)
    assert np.abs(jump[:, :, 1:]).max() < 1e-14
    assert -tab[0, 0, 0, -1] == pytest.approx(0.5, abs=1e-14)      # half filling
    tab2 = HC.hc_table(L, 1.0, beta, 0.2, 0.05, 0.3, 129)
    neg = np.array([((-(r % L)) % L) + L * ((-(r // L)) % L) for r in range(L * L)])
    assert np.abs(tab2[0, 1] - tab2[1, 0][neg]).max() < 1e-14
    assert np.abs(tab2[0, 0] - tab2[0, 0][neg]).max() < 1e-14
    # sum over cells of G(R, 0^-) = n_F(H(k = 0)), the k = 0 block, from the 2 x 2 matrix
    # exponential (mpmath, no eigendecomposition)
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    H0 = HC.hc_bloch(L, 1.0, 0.2, 0.05, 0.3)[0].real
    nF = mp.inverse(mp.expm(beta * mp.matrix(H0.tolist())) + mp.eye(2))
    total = -tab2[:, :, :, -1].sum(axis=2)
    for s in range(2):
        for t in range(2):
            assert total[s, t] == pytest.approx(float(nF[s, t]), abs=1e-13)
    # staggered field at half filling keeps one particle per cell
    tab3 = HC.hc_table(L, 1.0, beta, 0.0, 0.0, 0.4, 129)
    assert -tab3[0, 0, 0, -1] - tab3[1, 1, 0, -1] == pytest.approx(1.0, abs=1e-14)


def test_honeycomb_gather_layout():
    model = I.WORKLOADS["hc_su2_af_n8"].model
    small = I.HoneycombModel(4, model.t, model.beta, model.U, model.mu, model.alpha, model.delta, 65)
    tabs = HC.hc_model_tables(small)
    cfgs = I.make_configs(small, 3, 3, 1, 7)
    M4 = HC.hc_gather_one(tabs, cfgs.site, cfgs.tau, small.L, small.beta)
    assert M4.shape == (2, 3, 2, 3, 2)
    # diagonal blocks are equal-time (0^-) values: -G(beta^-) at R = 0
    for l in range(2):
        for s in range(2):
            for t in range(2):
                assert M4[l, 1, s, 1, t] == pytest.approx(-tabs[l, s, t, 0, -1], rel=1e-14)
    # the antiferromagnetic shift flips the sublattice roles between the spins
    assert small.sigma2[0] == pytest.approx(small.sigma2[1][::-1])
