"""CPU oracle for the connected-sum hot path of CoS++ (arXiv 2507.12349).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
timed CPU baseline of ``bench.py`` may import this package.  It shares no code
with the CUDA path; both read the seeded inputs of
``paper_2507_12349_b300.inputs`` and nothing else in common.

Functions and the passages they follow:

* ``brute``    -- sum over decorated covers, enumerated one by one (the
  definition of the connected sum, Results A: cycle covers, -1 and a flavor
  weight per closed loop, connectivity of the vertex graph).  n <= 5.
* ``closed``   -- determinants of every flavor block plus the subset
  subtraction c(S) = a(S) - sum c(T) a(S \\ T) of Methods A.  n <= 12.
* ``dp``       -- the merged clow-sequence DP of Results A / Alg. 2-3 in plain
  loops (``oracle_impl.h`` states each rule).  n <= 12.
* ``point_dp`` -- the unmerged point form of Alg. 2 (visited point set R, new
  heads at the smallest unvisited partner of a visited point), pure Python.
* ``propagators`` -- G0 tables by the plain momentum sum of Methods A, the
  linear interpolation in tau and the gather into M.
* ``torch_brute`` -- the brute-force sum as dense torch ops, for autograd.
* ``bip``      -- bipartite (two-sublattice) connected sums: the sum over every
  sublattice assignment of a single-assignment route (Methods A, strategy (i)),
  or the sublattice-resolved merged DP of Alg. 1-2 (``method="dp4"``).
* ``dp``, ``closed``, ``brute`` also take per-(flavor, vertex) shift weights
  (``sigma`` of shape [nf][n]).
* ``det_clow`` -- SU(2) connected sums with determinant weights by the DP without
  cycle factors of Alg. 1 (point-resolved states, interaction masks only, nonphysical
  clow sequences kept), on one or two sublattices (``oracle_det.h``).
* ``det_closed`` / ``det_brute`` -- the same sum from its definition: determinants of
  both spin blocks plus the subset subtraction of Methods A, or the block permutations
  enumerated one by one with a connectivity check.

Precision: 'd' (double), 'ld' (x87 long double) or 'q' (__float128).
"""
from __future__ import annotations

import ctypes
import itertools
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from . import build_oracle

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        dp_ = ctypes.POINTER(ctypes.c_double)
        for sfx in ("_d", "_ld", "_q"):
            f = getattr(L, "brute" + sfx)
            f.argtypes = [ctypes.c_int, ctypes.c_int, dp_, dp_, ctypes.c_int, dp_, dp_]
            f.restype = ctypes.c_int
            f = getattr(L, "closed" + sfx)
            f.argtypes = [ctypes.c_int, ctypes.c_int, dp_, dp_, dp_, dp_, dp_, dp_]
            f.restype = ctypes.c_int
            f = getattr(L, "dp" + sfx)
            f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp_, dp_, ctypes.c_int, dp_, dp_]
            f.restype = ctypes.c_int
            for name in ("brute_v",):
                f = getattr(L, name + sfx)
                f.argtypes = [ctypes.c_int, ctypes.c_int, dp_, dp_, ctypes.c_int, dp_, dp_]
                f.restype = ctypes.c_int
            f = getattr(L, "closed_v" + sfx)
            f.argtypes = [ctypes.c_int, ctypes.c_int, dp_, dp_, dp_, dp_, dp_, dp_]
            f.restype = ctypes.c_int
            f = getattr(L, "dp_v" + sfx)
            f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp_, dp_, ctypes.c_int, dp_, dp_]
            f.restype = ctypes.c_int
            f = getattr(L, "bip_sum" + sfx)
            f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp_, dp_, ctypes.c_int, ctypes.c_int, dp_, dp_]
            f.restype = ctypes.c_int
            f = getattr(L, "bip_dp4" + sfx)
            f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp_, dp_, ctypes.c_int, dp_, dp_]
            f.restype = ctypes.c_int
            f = getattr(L, "det_clow" + sfx)
            f.argtypes = [ctypes.c_int, ctypes.c_int, dp_, dp_, ctypes.c_int, dp_, dp_]
            f.restype = ctypes.c_int
            f = getattr(L, "dp_batch" + sfx)
            f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp_, dp_, ctypes.c_int,
                          dp_, dp_, ctypes.c_int]
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _sigma(sigma, nf: int, n: int):
    """Shift weights as a contiguous array and whether they are per (flavor, vertex):
    None, nf values (per flavor) or an [nf][n] array (per flavor and vertex)."""
    if sigma is None:
        return None, False
    sig = _f64(sigma)
    if sig.ndim == 2:
        if sig.shape != (nf, n):
            raise ValueError("per-vertex sigma must have shape [nf][n]")
        return np.ascontiguousarray(sig.ravel()), True
    return sig, False


def tiled(M: np.ndarray) -> np.ndarray:
    """Point matrices [nf][2n][2n] from vertex matrices [nf][n][n]: the
    2n x 2n matrix indexed by vertex = point mod n (Alg. 3's A_l indexing)."""
    M = np.asarray(M, dtype=np.float64)
    return np.ascontiguousarray(np.tile(M, (1, 2, 2)))


def brute(A_points: np.ndarray, sigma: Optional[Sequence[float]] = None, connected: bool = True,
          prec: str = "d") -> float:
    """Sum over (connected) decorated covers of 2n points, point matrices
    [nf][2n][2n]; sigma = per-flavor shift weights or None (no shift points)."""
    A = _f64(A_points)
    nf, np2, _ = A.shape
    n = np2 // 2
    sig, v = _sigma(sigma, nf, n)
    hi, lo = ctypes.c_double(), ctypes.c_double()
    rc = getattr(lib(), ("brute_v_" if v else "brute_") + prec)(n, nf, _ptr(A), _ptr(sig), int(connected),
                                          ctypes.byref(hi), ctypes.byref(lo))
    if rc:
        raise ValueError("brute: unsupported sizes")
    return hi.value + lo.value


def closed(M: np.ndarray, sigma: Optional[Sequence[float]] = None, prec: str = "d",
           subsets: bool = False):
    """Connected sum c(V) from determinants and the subset subtraction; with
    subsets=True also returns a(S) for every S and c(S) for every S containing
    vertex 0 (bit i of S = vertex i)."""
    M = _f64(M)
    nf, n, _ = M.shape
    sig, v = _sigma(sigma, nf, n)
    hi, lo = ctypes.c_double(), ctypes.c_double()
    a_all = np.zeros(1 << n) if subsets else None
    c_all = np.zeros(1 << n) if subsets else None
    rc = getattr(lib(), ("closed_v_" if v else "closed_") + prec)(n, nf, _ptr(M), _ptr(sig), ctypes.byref(hi), ctypes.byref(lo),
                                           _ptr(a_all), _ptr(c_all))
    if rc:
        raise ValueError("closed: unsupported sizes")
    if subsets:
        return hi.value + lo.value, a_all, c_all
    return hi.value + lo.value


def dp(M: np.ndarray, sigma: Optional[Sequence[float]] = None, weight: int = 1, absmode: bool = False,
       prec: str = "d", pair: bool = False):
    """Merged DP.  M [nf][n][n]; `weight` multiplies every closed loop (the
    symmetric SU(N) run passes one matrix and weight N)."""
    M = _f64(M)
    nf, n, _ = M.shape
    sig, v = _sigma(sigma, nf, n)
    hi, lo = ctypes.c_double(), ctypes.c_double()
    rc = getattr(lib(), ("dp_v_" if v else "dp_") + prec)(n, nf, int(weight), _ptr(M), _ptr(sig), int(absmode),
                                       ctypes.byref(hi), ctypes.byref(lo))
    if rc:
        raise ValueError("dp: unsupported sizes")
    return (hi.value, lo.value) if pair else hi.value + lo.value


def dp_batch(Ms: np.ndarray, sigma: Optional[Sequence[float]] = None, weight: int = 1,
             absmode: bool = False, prec: str = "d", nthreads: int = 0) -> Tuple[np.ndarray, np.ndarray, int]:
    """Merged DP over a batch [cfg][nf][n][n] of one order (OpenMP over
    configurations).  Returns (hi, lo, threads used)."""
    Ms = _f64(Ms)
    ncfg, nf, n, _ = Ms.shape
    sig = None if sigma is None else _f64(sigma)
    hi = np.zeros(ncfg)
    lo = np.zeros(ncfg)
    used = getattr(lib(), "dp_batch_" + prec)(ncfg, n, nf, int(weight), _ptr(Ms), _ptr(sig), int(absmode),
                                               _ptr(hi), _ptr(lo), int(nthreads))
    if used < 0:
        raise ValueError("dp_batch: unsupported sizes")
    return hi, lo, used


# ------------------------------------------------------------------ pure Python tiers

def brute_py(A_points: np.ndarray, sigma=None, connected: bool = True) -> float:
    """Second, independent brute force in pure Python (n <= 3): enumerate
    decorations, then permutations of the normal points; weight = product over
    cycles of (-sum_l prod A^l * prod of -sigma_l over shifts whose partner
    is on the cycle)."""
    A = np.asarray(A_points, dtype=np.float64)
    nf, np2, _ = A.shape
    n = np2 // 2
    total = 0.0
    decos = itertools.product(range(3), repeat=n) if sigma is not None else [(0,) * n]
    for deco in decos:
        shifts = {i if d == 1 else i + n for i, d in enumerate(deco) if d}
        pts = [p for p in range(np2) if p not in shifts]
        for img in itertools.permutations(pts):
            pi = dict(zip(pts, img))
            if connected:
                comp = {i: i for i in range(n)}

                def find(x):
                    while comp[x] != x:
                        x = comp[x]
                    return x
                for p in pts:
                    comp[find(p % n)] = find(pi[p] % n)
                if len({find(i) for i in range(n)}) > 1:
                    continue
            seen = set()
            w = 1.0
            for p in pts:
                if p in seen:
                    continue
                cyc = []
                q = p
                while q not in seen:
                    seen.add(q)
                    cyc.append(q)
                    q = pi[q]
                loop = 0.0
                for l in range(nf):
                    t = 1.0
                    for q in cyc:
                        t *= A[l, q, pi[q]]
                    for q in cyc:
                        if (q + n) % np2 in shifts:
                            t *= -sigma[l]
                    loop += t
                w *= -loop
            total += w
    return total


def point_dp(A_points: np.ndarray, weight: int = 1, connected: bool = True) -> float:
    """Unmerged point form of Alg. 2 (no sublattice labels, no shifts), pure
    Python.  States (u, v, R): head point u, current point v, visited point
    set R.  Extend: v -> w for every w not in R, weight A[v][w].  Close:
    weight -A[v][u] (times `weight`, Alg. 2's N_f); the next head is the
    smallest unvisited point whose partner is visited (connected=True, Results
    A / Alg. 2's P set) or simply the smallest unvisited point (connected=False,
    the Mahajan-Vinay head rule restricted to cycle covers).  With one matrix,
    weight 1 and connected=False the sum is det(A) (Results A)."""
    A = np.asarray(A_points, dtype=np.float64)
    np2 = A.shape[0]
    n = np2 // 2
    full = (1 << np2) - 1
    layer = {(0, 0, 1): 1.0}
    S = 0.0
    for _ in range(np2):
        nxt = {}
        for (u, v, R), w in layer.items():
            for x in range(np2):
                if not R & (1 << x):
                    key = (u, x, R | (1 << x))
                    nxt[key] = nxt.get(key, 0.0) + w * A[v, x]
            cw = -w * A[v, u] * weight
            if R == full:
                S += cw
                continue
            if connected:
                cand = [q for q in range(np2) if not R & (1 << q) and R & (1 << ((q + n) % np2))]
            else:
                cand = [q for q in range(np2) if not R & (1 << q)]
            if cand:
                h = min(cand)
                key = (h, h, R | (1 << h))
                nxt[key] = nxt.get(key, 0.0) + cw
        layer = nxt
    return S


def torch_brute(M, sigma=None):
    """Connected sum as dense torch ops over the enumerated connected
    decorated covers of the tiled matrix (n <= 3); differentiable in M
    [nf][n][n] and sigma [nf] (autograd reference for the adjoint)."""
    import torch
    nf, n, _ = M.shape
    np2 = 2 * n
    total = M.new_zeros(())
    decos = itertools.product(range(3), repeat=n) if sigma is not None else [(0,) * n]
    for deco in decos:
        shifts = {i if d == 1 else i + n for i, d in enumerate(deco) if d}
        pts = [p for p in range(np2) if p not in shifts]
        for img in itertools.permutations(pts):
            pi = dict(zip(pts, img))
            comp = {i: i for i in range(n)}

            def find(x):
                while comp[x] != x:
                    x = comp[x]
                return x
            for p in pts:
                comp[find(p % n)] = find(pi[p] % n)
            if len({find(i) for i in range(n)}) > 1:
                continue
            seen = set()
            w = M.new_ones(())
            for p in pts:
                if p in seen:
                    continue
                cyc = []
                q = p
                while q not in seen:
                    seen.add(q)
                    cyc.append(q)
                    q = pi[q]
                rows = torch.tensor([q % n for q in cyc])
                cols = torch.tensor([pi[q] % n for q in cyc])
                per_flavor = M[:, rows, cols].prod(dim=1)
                nsh = sum(1 for q in cyc if (q + n) % np2 in shifts)
                if nsh:
                    per_flavor = per_flavor * (-sigma) ** nsh
                w = w * (-per_flavor.sum())
            total = total + w
    return total


def bip(M4: np.ndarray, sigma2: Optional[np.ndarray] = None, weight: int = 1, absmode: bool = False,
        method: str = "sum_dp", prec: str = "d") -> float:
    """Bipartite connected sum.  M4 [nf][n][2][n][2] (flavor, vertex, sublattice, vertex,
    sublattice; sublattice 0 = A, 1 = B), sigma2 [nf][2] shift weights per flavor and
    sublattice, or None.  method: "sum_dp" / "sum_closed" / "sum_brute" = the sum over all
    2^n sublattice assignments of the merged DP / the closed form / brute force (the
    definition, Methods A strategy (i)); "dp4" = the sublattice-resolved merged DP of
    Alg. 1-2 (n <= 8)."""
    M4 = _f64(M4)
    nf, n = M4.shape[0], M4.shape[1]
    if M4.shape != (nf, n, 2, n, 2):
        raise ValueError("M4 must have shape [nf][n][2][n][2]")
    sig = None if sigma2 is None else _f64(sigma2).reshape(nf, 2)
    hi, lo = ctypes.c_double(), ctypes.c_double()
    if method == "dp4":
        rc = getattr(lib(), "bip_dp4_" + prec)(n, nf, int(weight), _ptr(M4), _ptr(sig), int(absmode),
                                               ctypes.byref(hi), ctypes.byref(lo))
    else:
        code = {"sum_dp": 0, "sum_closed": 1, "sum_brute": 2}[method]
        rc = getattr(lib(), "bip_sum_" + prec)(n, nf, int(weight), _ptr(M4), _ptr(sig), int(absmode), code,
                                               ctypes.byref(hi), ctypes.byref(lo))
    if rc:
        raise ValueError("bip: unsupported sizes or method")
    return hi.value + lo.value


def bip_assignment(M4: np.ndarray, sigma2: Optional[np.ndarray], s: Sequence[int]):
    """Vertex matrices [nf][n][n] and per-vertex shift weights [nf][n] of one sublattice
    assignment s (s_i in {0, 1})."""
    M4 = _f64(M4)
    s = np.asarray(s, dtype=np.int64)
    n = M4.shape[1]
    idx = np.arange(n)
    M = M4[:, idx[:, None], s[:, None], idx[None, :], s[None, :]]
    sig = None if sigma2 is None else _f64(sigma2)[:, s]
    return np.ascontiguousarray(M), sig


# ------------------------------------------------------------------ SU(2) determinant weights

def _det_blocks(G, alpha):
    """Spin blocks as [2][n][nsub][n][nsub] and diagonal shifts as [2][nsub]: G is [2][n][n]
    (one sublattice) or [2][n][2][n][2] (two)."""
    G = _f64(G)
    if G.ndim == 3 and G.shape[0] == 2 and G.shape[1] == G.shape[2]:
        n, nsub = G.shape[1], 1
        G = G.reshape(2, n, 1, n, 1)
    elif G.ndim == 5 and G.shape[0] == 2 and G.shape[2] == 2 and G.shape[4] == 2 and G.shape[1] == G.shape[3]:
        n, nsub = G.shape[1], 2
    else:
        raise ValueError("G must have shape [2][n][n] or [2][n][2][n][2]")
    al = None if alpha is None else _f64(alpha).reshape(2, nsub)
    return np.ascontiguousarray(G), al, n, nsub


def det_clow(G, alpha=None, absmode: bool = False, prec: str = "d") -> float:
    """Connected sum of an SU(2) model with determinant weights by the DP of Alg. 1.
    G [2][n][n] (spin up, spin down) or [2][n][2][n][2] (spin, vertex, sublattice, vertex,
    sublattice); alpha [2] or [2][2] diagonal shifts (a(p s, p s) - alpha_{spin, s}) or None."""
    Gb, al, n, nsub = _det_blocks(G, alpha)
    hi, lo = ctypes.c_double(), ctypes.c_double()
    rc = getattr(lib(), "det_clow_" + prec)(n, nsub, _ptr(Gb), _ptr(al), int(absmode), ctypes.byref(hi),
                                             ctypes.byref(lo))
    if rc:
        raise ValueError("det_clow: unsupported sizes")
    return hi.value + lo.value


def _det_assignment(Gb, al, n, nsub, S, s):
    """Shifted spin-block matrices restricted to the vertex list S with sublattices s."""
    mats = []
    for b in range(2):
        A = np.array([[Gb[b, i, s[x], j, s[y]] for y, j in enumerate(S)] for x, i in enumerate(S)])
        if al is not None:
            A = A - np.diag([al[b, s[x]] for x in range(len(S))])
        mats.append(A)
    return mats


def det_closed(G, alpha=None) -> float:
    """The connected sum from its definition (Methods A): a(S) = sum over sublattice
    assignments of det(A_up[S]) det(A_dn[S]) by LU, a(empty) = 1, and the subset subtraction
    c(S) = a(S) - sum_{T proper, T contains min S} c(T) a(S minus T).  n <= 10 (one
    sublattice) or n <= 7 (two)."""
    Gb, al, n, nsub = _det_blocks(G, alpha)
    if (nsub == 1 and n > 10) or (nsub == 2 and n > 7):
        raise ValueError("det_closed: n too large")
    a = np.zeros(1 << n)
    a[0] = 1.0
    for m in range(1, 1 << n):
        S = [i for i in range(n) if m >> i & 1]
        tot = 0.0
        for s in itertools.product(range(nsub), repeat=len(S)):
            up, dn = _det_assignment(Gb, al, n, nsub, S, s)
            tot += np.linalg.det(up) * np.linalg.det(dn)
        a[m] = tot
    c = np.zeros(1 << n)
    for m in range(1, 1 << n):
        low = m & -m
        rest = m ^ low
        val = a[m]
        t = rest
        while True:
            sub = t | low
            if sub != m:
                val -= c[sub] * a[m ^ sub]
            if t == 0:
                break
            t = (t - 1) & rest
        c[m] = val
    return float(c[(1 << n) - 1])


def det_brute(G, alpha=None) -> float:
    """The connected sum diagram by diagram (n <= 4): every pair of permutations (one per
    spin block) and sublattice assignment, signed by sgn(pi_up) sgn(pi_dn), kept when the
    vertices joined by i - pi_b(i) form one component."""
    Gb, al, n, nsub = _det_blocks(G, alpha)
    if n > 4:
        raise ValueError("det_brute: n <= 4")

    def sign(p):
        sg, seen = 1, [False] * n
        for i in range(n):
            if seen[i]:
                continue
            j, ln = i, 0
            while not seen[j]:
                seen[j] = True
                j = p[j]
                ln += 1
            sg *= -1 if ln % 2 == 0 else 1
        return sg

    perms = list(itertools.permutations(range(n)))
    total = 0.0
    for s in itertools.product(range(nsub), repeat=n):
        up, dn = _det_assignment(Gb, al, n, nsub, list(range(n)), s)
        for pu in perms:
            wu = sign(pu) * np.prod([up[i, pu[i]] for i in range(n)])
            for pd in perms:
                comp = list(range(n))

                def find(x):
                    while comp[x] != x:
                        x = comp[x]
                    return x
                for i in range(n):
                    comp[find(i)] = find(pu[i])
                    comp[find(i)] = find(pd[i])
                if len({find(i) for i in range(n)}) > 1:
                    continue
                total += wu * sign(pd) * np.prod([dn[i, pd[i]] for i in range(n)])
    return total
