"""CPU-side checks of the C ABI: the library builds, loads, exports every
declared symbol, rejects bad arguments without a device, and its host-built
DP structure has the counts of the merged recurrence."""
import itertools
import os
import re

import pytest

from paper_2507_12349_b300 import binding as B
from paper_2507_12349_b300 import build as BLD

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cos.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(cos_\w+)\s*\(", src, flags=re.M)))


def prob(lattice, weights, precision, n_cfg, n_max, order=None, tables=None, offset=None, site=None, tau=None,
         moff=None, M=None, n_mat=0, wt=0, shift=None):
    """A raw cos_problem with integer device addresses (for argument checks without a device)."""
    import ctypes
    p = B.cos_problem()
    p.lattice, p.weights, p.precision, p.n_cfg, p.n_max = lattice, weights, precision, n_cfg, n_max
    p.d_order, p.tables, p.d_offset, p.d_site, p.d_tau, p.d_moff, p.d_M = order, tables, offset, site, tau, moff, M
    p.n_mat, p.loop_weight = n_mat, wt
    if shift is not None:
        p.h_shift = ctypes.cast(shift, ctypes.POINTER(ctypes.c_double))
    return p


def test_library_builds_and_exports_every_declared_symbol():
    lib = B.lib()
    decl = declared_functions()
    assert decl, "no declarations parsed"
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(decl) == sorted(B.EXPORTS)


def test_build_targets_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(BLD.ARCH)


def test_argument_errors_are_synchronous():
    lib = B.lib()
    import ctypes
    # order out of range is rejected before any device work
    rc = lib.cos_connected_sum_matrices(1, 13, None, None, 1, 1, None, None, 0, None, None, None)
    assert rc == -2
    rc = lib.cos_connected_sum_matrices(-1, 4, None, None, 1, 1, None, None, 0, None, None, None)
    assert rc == -1
    rc = lib.cos_connected_sum_matrices(1, 4, None, None, 9, 1, None, None, 0, None, None, None)
    assert rc == -1
    rc = lib.cos_connected_sum_matrices(1, 4, None, None, 1, 1, None, None, 7, None, None, None)
    assert rc == -1
    # empty batch is a no-op
    assert lib.cos_connected_sum_matrices(0, 4, None, None, 1, 1, None, None, 0, None, None, None) == 0
    # all-subsets mode: a(S) needs every root; all_roots is a flag
    fake = 256                                          # never dereferenced: rejected before any launch
    assert lib.cos_subsets(ctypes.byref(prob(0, 0, 0, 1, 4, n_mat=1, wt=1)), 1, None, None, None) == -1
    assert lib.cos_subsets(ctypes.byref(prob(0, 0, 0, 1, 4, fake, moff=fake, M=fake, n_mat=1, wt=1)), 0, fake, fake,
                           None) == -1
    assert lib.cos_subsets(ctypes.byref(prob(0, 0, 0, 1, 4, fake, moff=fake, M=fake, n_mat=1, wt=1)), 2, fake, None,
                           None) == -1
    assert lib.cos_subsets(ctypes.byref(prob(0, 0, 0, 0, 4, n_mat=1, wt=1)), 1, None, None, None) == 0
    # descriptor calls (cos_problem): determinant weights, bipartite lattices, gradients, subsets
    fw = lambda p, out=None: lib.cos_forward(ctypes.byref(p), out, None, None)
    gr = lambda p, gout=None, **k: lib.cos_grad(ctypes.byref(p), gout, None, k.get("gM"), k.get("gmoff"),
                                                k.get("gshift"), k.get("gmu"), k.get("galpha"), None)
    ss = lambda p, roots, c, a=None: lib.cos_subsets(ctypes.byref(p), roots, c, a, None)
    assert lib.cos_forward(None, None, None, None) == -1
    assert fw(prob(5, 0, 0, 1, 4, fake, moff=fake, M=fake), fake) == -1            # unknown lattice
    assert fw(prob(0, 7, 0, 1, 4, fake, moff=fake, M=fake), fake) == -1            # unknown weight kind
    # square determinant weights: orders up to 12
    assert fw(prob(0, 1, 0, 1, 13)) == -2
    assert fw(prob(0, 1, 0, 1, 4)) == -1
    assert fw(prob(0, 1, 9, 1, 4, fake, moff=fake, M=fake), fake) == -1           # bad precision
    assert fw(prob(0, 1, 0, 0, 4)) == 0
    # bipartite determinant weights: orders up to 9
    assert fw(prob(1, 1, 0, 1, 10, fake, moff=fake, M=fake), fake) == -2
    assert fw(prob(1, 1, 7, 1, 4, fake, moff=fake, M=fake), fake) == -1
    assert fw(prob(1, 1, 0, 1, 4)) == -1
    # loop weights from coordinates take their shifts from the tables (never dereferenced here)
    sh = (ctypes.c_double * 4)(0.1, 0.2, 0.3, 0.4)
    assert fw(prob(0, 0, 0, 1, 4, fake, tables=fake, offset=fake, site=fake, tau=fake, shift=sh), fake) == -1
    # gradients: FP64 only; the coordinates and matrices forms take their own outputs
    assert gr(prob(0, 0, 1, 1, 4, fake, moff=fake, M=fake, n_mat=1, wt=1), fake) == -6
    assert gr(prob(0, 0, 0, 1, 4, fake, tables=fake, offset=fake, site=fake, tau=fake), fake, gshift=fake) == -1
    assert gr(prob(0, 1, 0, 1, 4, fake, tables=fake, offset=fake, site=fake, tau=fake), fake, galpha=fake) == -1
    assert gr(prob(0, 0, 0, 1, 4, fake, moff=fake, M=fake, n_mat=1, wt=1), fake, gmoff=fake) == -1
    assert gr(prob(0, 1, 0, 1, 13)) == -2
    assert gr(prob(0, 1, 0, 1, 4)) == -1
    assert gr(prob(0, 1, 0, 0, 4)) == 0
    assert gr(prob(1, 0, 0, 1, 10, fake, moff=fake, M=fake, n_mat=2, wt=1), fake) == -2
    assert gr(prob(1, 1, 0, 0, 4)) == 0
    # every subset: explicit matrices only; bipartite orders up to 9, FP64; all_roots 0 or 1
    assert ss(prob(0, 0, 0, 1, 4, fake, tables=fake, offset=fake, site=fake, tau=fake), 1, fake) == -6
    assert ss(prob(1, 0, 0, 1, 10, fake, moff=fake, M=fake, n_mat=1, wt=1), 1, fake) == -2
    assert ss(prob(1, 0, 1, 1, 4, fake, moff=fake, M=fake, n_mat=1, wt=1), 1, fake) == -6
    assert ss(prob(1, 0, 0, 1, 4, fake, moff=fake, M=fake, n_mat=1, wt=1), 2, fake) == -1
    assert ss(prob(1, 0, 0, 1, 4, fake, moff=fake, M=fake, n_mat=1, wt=1), 0, fake, fake) == -1
    assert ss(prob(1, 0, 0, 0, 4, n_mat=1, wt=1), 1, None) == 0
    assert ss(prob(1, 1, 2, 1, 4, fake, moff=fake, M=fake), 1, fake) == -6
    assert ss(prob(1, 1, 0, 1, 4), 1, None) == -1
    assert ss(prob(0, 1, 1, 1, 4, fake, moff=fake, M=fake), 1, fake) == -6
    assert ss(prob(0, 1, 0, 1, 4, fake, moff=fake, M=fake), 0, fake, fake) == -1
    assert lib.cos_status_string(-2) == b"order out of range"
    inf = B.cos_structure_info()
    assert lib.cos_structure(0, ctypes.byref(inf)) == -2


def count_merged(n):
    """Independent count of masks, slots, reachable states and multiply-adds."""
    masks = slots = states = ext = close = shift = 0
    for mu in itertools.product(range(3), repeat=n):
        if mu[0] == 0:
            continue
        masks += 1
        A = [i for i in range(n) if mu[i] >= 1]
        ones = [i for i in range(n) if mu[i] == 1]
        B_ = [i for i in range(n) if mu[i] == 2]
        H = [0] if mu[0] == 1 else B_
        J = [j for j in range(n) if mu[j] <= 1]
        Z = [j for j in range(n) if mu[j] == 0]
        need = bool(ones) or len(B_) == n
        slots += len(H) * len(A)
        for h in H:
            if h == 0 and mu[0] == 1:
                V = [0] if len(A) == 1 else [v for v in A if v]
            elif h == 0:
                V = A
            else:
                V = [v for v in A if v and not (v == h and any(o < h for o in ones))]
            states += len(V)
            ext += len(V) * len(J)
            close += len(V) if need else 0
            shift += len(Z)
    return masks, slots, states, ext, close, shift


@pytest.mark.parametrize("n", [1, 2, 4, 7, 8])
def test_structure_counts(n):
    inf = B.cos_structure(n)
    assert (inf.masks, inf.slots, inf.states, inf.fma_ext, inf.fma_close, inf.mul_shift) == count_merged(n)
    assert inf.masks == 2 * 3 ** (n - 1)


def test_structure_counts_large_orders():
    # slot counts of the merged state space: 252 at n = 4, 708588 at n = 10, 8581788 at n = 12
    assert B.cos_structure(4).slots == 252
    assert B.cos_structure(10).slots == 708588
    inf = B.cos_structure(12)
    assert inf.slots == 8581788 and inf.max_layer_slots == 1262547


def test_binding_wraps_every_entry_point():
    """Every exported call has a same-named Python wrapper (or a method of the object
    it manages: Tables for table calls, Plan for plan calls)."""
    methods = {"cos_free_tables": (B.Tables, "close"), "cos_get_tables_info": (B.Tables, "info"),
               "cos_copy_table": (B.Tables, "table"), "cos_plan_launch": (B.Plan, "launch"),
               "cos_plan_status": (B.Plan, "status"), "cos_plan_grid": (B.Plan, "grid"),
               "cos_plan_destroy": (B.Plan, "close"), "cos_status_string": (B, "STATUS"),
               "cos_last_error": (B, "_check")}
    for name in B.EXPORTS:
        if name in methods:
            owner, attr = methods[name]
            assert hasattr(owner, attr), name
        else:
            assert callable(getattr(B, name, None)), name


def count_bipartite(n):
    """Independent count of the bipartite structure: masks in {0, 1A, 1B, 2}^n with vertex 0
    visited, rows (h, s_h) -- one for the first loop's head, else two -- and reachable
    endpoint states (one for a half-visited endpoint or v = h, else two sublattices)."""
    full = (1 << n) - 1
    masks = slots = states = ext = close = 0
    for d in itertools.product(range(4), repeat=n):
        if d[0] == 0:
            continue
        masks += 1
        A = sum(1 << i for i in range(n) if d[i] > 0)
        B = sum(1 << i for i in range(n) if d[i] == 3)
        ones = A & ~B
        H = [0] if ones & 1 else [i for i in range(n) if B >> i & 1]
        slots += 4 * len(H) * bin(A).count("1")
        T = sum(2 if d[j] == 0 else 1 for j in range(n) if d[j] != 3)
        need = ones != 0 or B == full
        for h in H:
            rows = 1 if (h == 0 and ones & 1) else 2
            if h == 0 and ones & 1:
                V = [0] if A == 1 else [v for v in range(1, n) if A >> v & 1]
            elif h == 0:
                V = [v for v in range(n) if A >> v & 1]
            else:
                V = [v for v in range(1, n) if A >> v & 1
                     and not (v == h and any(ones >> o & 1 for o in range(h)))]
            nv = sum(1 if (ones >> v & 1 or v == h) else 2 for v in V)
            states += rows * nv
            ext += rows * nv * T
            close += rows * nv if need else 0
    return masks, slots, states, ext, close


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_bipartite_structure_counts(n):
    inf = B.cos_bipartite_structure(n)
    masks, slots, states, ext, close = count_bipartite(n)
    assert (inf.masks, inf.slots, inf.states, inf.fma_ext, inf.fma_close) == (masks, slots, states, ext, close)


def test_bipartite_argument_errors():
    lib = B.lib()
    import ctypes
    fake = 256     # never dereferenced: rejected before any launch
    fw = lambda p: lib.cos_forward(ctypes.byref(p), fake, None, None)
    assert fw(prob(1, 0, 0, 1, 10, fake, moff=fake, M=fake, n_mat=1, wt=1)) == -2
    assert fw(prob(1, 0, 7, 1, 4, fake, moff=fake, M=fake, n_mat=1, wt=1)) == -1
    assert fw(prob(1, 0, 0, 1, 4, None, moff=fake, M=fake, n_mat=1, wt=1)) == -1
    assert lib.cos_forward(ctypes.byref(prob(1, 0, 0, 0, 4, n_mat=1, wt=1)), None, None, None) == 0
    inf = B.cos_structure_info()
    assert lib.cos_bipartite_structure(10, ctypes.byref(inf)) == -2


def test_instrument_library_exports_and_rejects_bad_arguments():
    """The benchmark's instruments live in their own library (not libcos): it loads without a
    device, exports its three entry points, and turns bad arguments into -1 before any launch."""
    L = B.instr_lib()
    for name in ("cos_instr_fma_probe", "cos_instr_row_traffic", "cos_instr_convert_check"):
        assert hasattr(L, name), name
        assert not hasattr(B.lib(), name), name
    assert L.cos_instr_fma_probe(9, 1, 32, 1, 8, None) == -1          # unknown kind
    assert L.cos_instr_fma_probe(0, 1, 16, 1, 8, None) == -1          # fewer than a warp
    assert L.cos_instr_row_traffic(3, 1, 1, 32, 1, 8, 8, 1, None) == -1   # unknown mode
    assert L.cos_instr_row_traffic(0, 2, 1, 32, 1, 8, 8, 1, None) == -1   # unsupported rows in flight
    assert L.cos_instr_row_traffic(0, 1, 1, 32, 1, 8, 8, 0, None) == -1   # no rows
    assert L.cos_instr_row_traffic(0, 1, 1, 32, 1, None, 8, 1, None) == -1
    assert L.cos_instr_convert_check(-1, None, None, None, None, None) == -1
