"""Pins of the SU(2) determinant-weight oracle (the DP without cycle factors, Alg. 1).

Each check compares `det_clow` with something other than itself:
  * the definition: LU determinants of both spin blocks plus the subset subtraction of
    Methods A (`det_closed`), and the block permutations enumerated one by one with a
    connectivity check (`det_brute`), on one and two sublattices, with diagonal shifts;
  * the subset exponential: det(A_up) det(A_dn) by LU equals the sum over set partitions of
    the vertices of the product of `det_clow` of each block (vertex 0's block enumerated);
  * the CoS relation: with two flavors, loop weight 1 and no shift points every vertex sends
    one point to each flavor in 2 ways, so the merged CoS DP (itself pinned against brute
    force and LU) equals 2^n times the determinant-weight sum, also per sublattice sum;
  * n = 1 closed form; a vertex with no propagator to the others makes the sum vanish;
  * invariances: transposition, vertex relabeling (the head rule), spin swap, sublattice
    swap, homogeneity c(t G, t alpha) = t^(2n) c(G, alpha); the mass bounds |c|;
  * c is linear in every single matrix entry (an entry occurs at most once in a determinant
    term and in one factor of each subtraction product): second differences vanish, while
    a diagonal shift alpha (a whole diagonal at once) is not linear.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2507_12349_b300 import inputs as I


def rand_g(seed, n, nsub, scale=0.9):
    M = I.random_matrices(seed, 1, 2, nsub * n, scale)[0]        # [2][n nsub][n nsub], index i nsub + s
    return np.ascontiguousarray(M if nsub == 1 else M.reshape(2, n, 2, n, 2))


def rand_alpha(seed, nsub):
    return I.random_matrices(seed + 555, 1, 1, 2 * nsub, 0.3)[0, 0, 0][: 2 * nsub].reshape(2, nsub)


def mass(G, al=None):
    return O.det_clow(G, al, absmode=True)


@pytest.mark.parametrize("nsub,n", [(1, 1), (1, 2), (1, 3), (1, 4), (2, 1), (2, 2), (2, 3), (2, 4)])
def test_det_clow_matches_closed_and_brute(nsub, n):
    G = rand_g(100 * nsub + n, n, nsub)
    al = rand_alpha(n, nsub)
    for a in (None, al):
        ref = O.det_clow(G, a, prec="q")
        tol = 1e-13 * mass(G, a)
        assert O.det_closed(G, a) == pytest.approx(ref, abs=tol)
        assert O.det_brute(G, a) == pytest.approx(ref, abs=tol)
        assert O.det_clow(G, a, prec="d") == pytest.approx(ref, abs=tol)


@pytest.mark.parametrize("nsub,n", [(1, 6), (1, 8), (2, 5), (2, 6)])
def test_det_clow_matches_closed_larger(nsub, n):
    G = rand_g(7 * n + nsub, n, nsub)
    al = rand_alpha(2 * n, nsub)
    ref = O.det_clow(G, al, prec="ld")
    assert O.det_closed(G, al) == pytest.approx(ref, abs=1e-12 * mass(G, al))


@pytest.mark.parametrize("nsub,n", [(1, 5), (2, 4)])
def test_subset_exponential_against_lu(nsub, n):
    """a(V) = sum over set partitions of V of prod c(block): enumerate vertex 0's block T
    and recurse on the rest, with every c from det_clow on the sub-matrices."""
    G = rand_g(40 + n, n, nsub)
    al = rand_alpha(9, nsub)

    def sub(S):
        S = list(S)
        if nsub == 1:
            return G[:, S][:, :, S]
        return G[:, S][:, :, :, S]

    def a_of(S):
        if not S:
            return 1.0
        first, rest = S[0], S[1:]
        tot = 0.0
        for r in range(len(rest) + 1):
            for T in itertools.combinations(rest, r):
                blk = (first,) + T
                tot += O.det_clow(sub(blk), al, prec="q") * a_of(tuple(x for x in rest if x not in T))
        return tot

    lu = 0.0
    for s in itertools.product(range(nsub), repeat=n):
        mats = []
        for b in range(2):
            if nsub == 1:
                A = G[b].copy()
            else:
                A = np.array([[G[b, i, s[i], j, s[j]] for j in range(n)] for i in range(n)])
            mats.append(A - np.diag([al[b, s[i] if nsub == 2 else 0] for i in range(n)]))
        lu += np.linalg.det(mats[0]) * np.linalg.det(mats[1])
    assert a_of(tuple(range(n))) == pytest.approx(lu, rel=1e-11, abs=1e-13)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 10])
def test_cos_relation_square(n):
    G = rand_g(300 + n, n, 1)
    ref = O.dp(G, None, weight=1, prec="ld")
    got = O.det_clow(G, prec="ld")
    assert 2.0 ** n * got == pytest.approx(ref, abs=1e-13 * 2.0 ** n * mass(G))


@pytest.mark.parametrize("n", [1, 3, 5, 7])
def test_cos_relation_bipartite(n):
    G = rand_g(400 + n, n, 2)
    ref = O.bip(G, None, weight=1, method="dp4" if n <= 8 else "sum_dp", prec="ld")
    got = O.det_clow(G, prec="ld")
    assert 2.0 ** n * got == pytest.approx(ref, abs=1e-13 * 2.0 ** n * mass(G))


def test_order_one_closed_form():
    for nsub in (1, 2):
        G = rand_g(5 + nsub, 1, nsub)
        al = rand_alpha(1, nsub)
        g = G.reshape(2, nsub, nsub)
        ref = sum((g[0, s, s] - al[0, s]) * (g[1, s, s] - al[1, s]) for s in range(nsub))
        assert O.det_clow(G, al, prec="q") == pytest.approx(ref, rel=1e-15)
        m = sum((abs(g[0, s, s]) + abs(al[0, s])) * (abs(g[1, s, s]) + abs(al[1, s])) for s in range(nsub))
        assert mass(G, al) == pytest.approx(m, rel=1e-15)


@pytest.mark.parametrize("nsub", [1, 2])
def test_isolated_vertex_gives_zero(nsub):
    n = 5
    G = rand_g(77, n, nsub).copy()
    for iso in (0, 3):
        H = G.copy()
        if nsub == 1:
            keep = H[:, iso, iso].copy()
            H[:, iso, :] = 0.0
            H[:, :, iso] = 0.0
            H[:, iso, iso] = keep
        else:
            keep = H[:, iso, :, iso, :].copy()
            H[:, iso, :, :, :] = 0.0
            H[:, :, :, iso, :] = 0.0
            H[:, iso, :, iso, :] = keep
        assert O.det_clow(H, prec="q") == pytest.approx(0.0, abs=1e-15 * mass(H))


@pytest.mark.parametrize("nsub,n", [(1, 7), (2, 6)])
def test_invariances(nsub, n):
    G = rand_g(900 + n, n, nsub)
    al = rand_alpha(4, nsub)
    ref = O.det_clow(G, al, prec="ld")
    tol = 1e-13 * mass(G, al)
    # transposition of both blocks
    GT = np.ascontiguousarray(np.swapaxes(G, 1, 2) if nsub == 1 else G.transpose(0, 3, 4, 1, 2))
    assert O.det_clow(GT, al, prec="ld") == pytest.approx(ref, abs=tol)
    # vertex relabeling
    perm = np.random.default_rng(n).permutation(n)
    GP = G[:, perm][:, :, perm] if nsub == 1 else G[:, perm][:, :, :, perm]
    assert O.det_clow(np.ascontiguousarray(GP), al, prec="ld") == pytest.approx(ref, abs=tol)
    # spin swap
    assert O.det_clow(np.ascontiguousarray(G[::-1]), al[::-1], prec="ld") == pytest.approx(ref, abs=tol)
    # sublattice relabeling A <-> B
    if nsub == 2:
        GS = np.ascontiguousarray(G[:, :, ::-1, :, ::-1])
        assert O.det_clow(GS, al[:, ::-1], prec="ld") == pytest.approx(ref, abs=tol)
    # homogeneity
    t = 1.3
    assert O.det_clow(t * G, t * al, prec="ld") == pytest.approx(t ** (2 * n) * ref, abs=t ** (2 * n) * tol)
    assert abs(ref) <= mass(G, al) * (1 + 1e-12)


@pytest.mark.parametrize("nsub", [1, 2])
def test_linear_in_every_entry(nsub):
    n = 4 if nsub == 1 else 3
    G = rand_g(71 + nsub, n, nsub)
    al = rand_alpha(8, nsub)
    scale = mass(G, al)
    rng = np.random.default_rng(nsub)
    for _ in range(6):
        idx = tuple(int(rng.integers(s)) for s in G.shape)
        v = []
        for h in (-1.0, 0.0, 1.0):
            Gp = G.copy(); Gp[idx] += h
            v.append(O.det_clow(Gp, al, prec="q"))
        assert abs(v[0] - 2 * v[1] + v[2]) <= 1e-14 * scale, idx
    v = []
    for h in (-1.0, 0.0, 1.0):
        a2 = al.copy(); a2[0, 0] += h
        v.append(O.det_clow(G, a2, prec="q"))
    assert abs(v[0] - 2 * v[1] + v[2]) > 1e-6 * abs(v[1])
