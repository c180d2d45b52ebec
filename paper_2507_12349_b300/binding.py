"""ctypes binding of libcos (include/cos.h): same names, argument marshalling only.

Every step of the connected-sum path runs in the CUDA kernels of libcos.so; this
module only converts torch tensors to device pointers and the current CUDA
stream to a handle.  There is no host fallback: if the library or a CUDA device
is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

COS_NMAX = 12
COS_MAX_FLAVORS = 8
COS_FP64 = 0
COS_MIXED = 1
COS_DF64 = 2
PRECISIONS = {"fp64": COS_FP64, "mixed": COS_MIXED, "df64": COS_DF64}

STATUS = {0: "COS_OK", -1: "COS_ERR_ARG", -2: "COS_ERR_ORDER", -3: "COS_ERR_CUDA", -4: "COS_ERR_TIMEOUT",
          -5: "COS_ERR_NONFINITE", -6: "COS_ERR_UNIMPLEMENTED", -7: "COS_ERR_NOMEM"}

# Every symbol include/cos.h declares (checked by the CPU tests).
EXPORTS = [
    "cos_build_propagators", "cos_free_tables", "cos_get_tables_info", "cos_copy_table", "cos_gather",
    "cos_connected_sum_matrices", "cos_connected_sum_matrices_noalloc", "cos_connected_sum_batch",
    "cos_build_propagators_honeycomb", "cos_gather_bipartite", "cos_bipartite_structure",
    "cos_forward", "cos_grad", "cos_subsets",
    "cos_connected_sum_grad", "cos_grad_checkpoint_plan", "cos_sync_status", "cos_release_workspace",
    "cos_status_string",
    "cos_last_error", "cos_structure",
    "cos_plan_create_batch", "cos_plan_create_matrices", "cos_plan_launch", "cos_plan_status", "cos_plan_grid",
    "cos_plan_destroy", "cos_set_tuning", "cos_get_tuning", "cos_autotune",
]


class CosError(RuntimeError):
    def __init__(self, status: int, where: str, message: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} {message}".strip())


class cos_model(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("t", ctypes.c_double), ("beta", ctypes.c_double), ("U", ctypes.c_double),
                ("n_flavors", ctypes.c_int), ("mu", ctypes.POINTER(ctypes.c_double)),
                ("alpha", ctypes.POINTER(ctypes.c_double)), ("n_tau", ctypes.c_int)]


class cos_tables_info(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("n_tau", ctypes.c_int), ("n_flavors", ctypes.c_int),
                ("symmetric", ctypes.c_int), ("n_mat", ctypes.c_int), ("beta", ctypes.c_double),
                ("U", ctypes.c_double), ("sigma", ctypes.c_double * COS_MAX_FLAVORS),
                ("d_G", ctypes.c_void_p), ("d_dGdmu", ctypes.c_void_p), ("bipartite", ctypes.c_int),
                ("sigma2", (ctypes.c_double * 2) * COS_MAX_FLAVORS)]


class cos_honeycomb_model(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("t", ctypes.c_double), ("beta", ctypes.c_double), ("U", ctypes.c_double),
                ("n_flavors", ctypes.c_int), ("mu", ctypes.POINTER(ctypes.c_double)),
                ("alpha", ctypes.POINTER(ctypes.c_double)), ("delta", ctypes.POINTER(ctypes.c_double)),
                ("n_tau", ctypes.c_int)]


class cos_structure_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("masks", ctypes.c_int64), ("slots", ctypes.c_int64),
                ("max_layer_slots", ctypes.c_int64), ("states", ctypes.c_int64), ("fma_ext", ctypes.c_int64),
                ("fma_close", ctypes.c_int64), ("mul_shift", ctypes.c_int64)]


_lib = None


TUNING_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_b300.txt")


COS_SQUARE, COS_BIPARTITE = 0, 1
COS_LOOPS, COS_DETERMINANTS = 0, 1


class cos_problem(ctypes.Structure):
    """include/cos.h cos_problem: lattice, weight kind, precision, and the input (vertex
    coordinates with tables, or explicit matrices)."""
    _fields_ = [("lattice", ctypes.c_int), ("weights", ctypes.c_int), ("precision", ctypes.c_int),
                ("n_cfg", ctypes.c_int), ("n_max", ctypes.c_int), ("d_order", ctypes.c_void_p),
                ("tables", ctypes.c_void_p), ("d_offset", ctypes.c_void_p), ("d_site", ctypes.c_void_p),
                ("d_tau", ctypes.c_void_p), ("d_moff", ctypes.c_void_p), ("d_M", ctypes.c_void_p),
                ("n_mat", ctypes.c_int), ("loop_weight", ctypes.c_int),
                ("h_shift", ctypes.POINTER(ctypes.c_double))]


def lib(build: bool = True):
    """Load libcos.so (building it from source first if it is missing or stale)."""
    global _lib
    if _lib is None:
        if "COS_TUNE_FILE" not in os.environ and os.path.exists(TUNING_FILE):
            os.environ["COS_TUNE_FILE"] = TUNING_FILE
        path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise OSError(f"libcos.so not found at {path}; run paper_2507_12349_b300.build")
        L = ctypes.CDLL(path)
        vp, i32, i64, dptr = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        L.cos_build_propagators.argtypes = [ctypes.POINTER(cos_model), vp, ctypes.POINTER(vp)]
        L.cos_free_tables.argtypes = [vp]
        L.cos_get_tables_info.argtypes = [vp, ctypes.POINTER(cos_tables_info)]
        L.cos_copy_table.argtypes = [vp, i32, vp, vp]
        L.cos_gather.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp]
        L.cos_connected_sum_matrices.argtypes = [i32, i32, vp, vp, i32, i32, dptr, vp, i32, vp, vp, vp]
        L.cos_connected_sum_matrices_noalloc.argtypes = [i32, i32, vp, vp, i32, i32, dptr, vp, i32, vp, vp, vp]
        pp = ctypes.POINTER(cos_problem)
        L.cos_forward.argtypes = [pp, vp, vp, vp]
        L.cos_grad.argtypes = [pp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.cos_subsets.argtypes = [pp, i32, vp, vp, vp]
        L.cos_build_propagators_honeycomb.argtypes = [ctypes.POINTER(cos_honeycomb_model), vp, ctypes.POINTER(vp)]
        L.cos_gather_bipartite.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp]
        L.cos_bipartite_structure.argtypes = [i32, ctypes.POINTER(cos_structure_info)]
        L.cos_connected_sum_grad.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.cos_connected_sum_batch.argtypes = [vp, i32, i32, vp, vp, vp, vp, i32, vp, vp, vp]
        L.cos_sync_status.argtypes = [vp]
        L.cos_release_workspace.argtypes = [vp]
        L.cos_status_string.argtypes = [i32]
        L.cos_status_string.restype = ctypes.c_char_p
        L.cos_last_error.argtypes = []
        L.cos_last_error.restype = ctypes.c_char_p
        L.cos_structure.argtypes = [i32, ctypes.POINTER(cos_structure_info)]
        L.cos_grad_checkpoint_plan.argtypes = [i32, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint32),
                                               ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.cos_plan_create_batch.argtypes = [vp, i32, i32, vp, vp, vp, vp, i32, vp, vp, vp, ctypes.POINTER(vp)]
        L.cos_plan_create_matrices.argtypes = [i32, i32, vp, vp, i32, i32, dptr, vp, i32, vp, vp, vp,
                                               ctypes.POINTER(vp)]
        L.cos_plan_launch.argtypes = [vp, vp]
        L.cos_plan_status.argtypes = [vp, vp]
        L.cos_plan_grid.argtypes = [vp, ctypes.POINTER(i32)]
        L.cos_plan_destroy.argtypes = [vp]
        L.cos_set_tuning.argtypes = [i32, i32, i32, i32, i32, i32]
        L.cos_get_tuning.argtypes = [i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.cos_autotune.argtypes = [i32, i32, i32, i32, i32, i32, vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                   ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]
        for name in EXPORTS:
            f = getattr(L, name)
            if name not in ("cos_status_string", "cos_last_error"):
                f.restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != 0:
        raise CosError(rc, where, lib().cos_last_error().decode())


def _stream(stream=None) -> ctypes.c_void_p:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, dtype=None) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None:
        import torch
        want = {"f64": torch.float64, "i32": torch.int32, "i64": torch.int64}[dtype]
        if t.dtype != want:
            raise TypeError(f"expected {want}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


class Tables:
    """Owner of device propagator tables (cos_build_propagators / cos_free_tables)."""

    def __init__(self, handle: ctypes.c_void_p):
        self.handle = handle

    def info(self) -> cos_tables_info:
        inf = cos_tables_info()
        _check(lib().cos_get_tables_info(self.handle, ctypes.byref(inf)), "cos_get_tables_info")
        return inf

    def table(self, deriv: bool = False, stream=None):
        """Device copy of the table [n_mat][L^2][n_tau] (G0, or dG0/dmu with deriv=True);
        honeycomb tables: [n_mat][2][2][L^2][n_tau]."""
        import torch
        inf = self.info()
        blocks = 4 if inf.bipartite else 1
        buf = torch.empty(inf.n_mat * blocks * inf.L * inf.L * inf.n_tau, dtype=torch.float64, device="cuda")
        _check(lib().cos_copy_table(self.handle, int(deriv), _ptr(buf), _stream(stream)), "cos_copy_table")
        if inf.bipartite:
            return buf.view(inf.n_mat, 2, 2, inf.L * inf.L, inf.n_tau)
        return buf.view(inf.n_mat, inf.L * inf.L, inf.n_tau)

    def close(self):
        if self.handle:
            lib().cos_free_tables(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cos_build_propagators(L: int, t: float, beta: float, U: float, mu: Sequence[float], alpha: Sequence[float],
                          n_tau: int, stream=None) -> Tables:
    mu_a = (ctypes.c_double * len(mu))(*mu)
    al_a = (ctypes.c_double * len(alpha))(*alpha)
    m = cos_model(int(L), float(t), float(beta), float(U), len(mu), mu_a, al_a, int(n_tau))
    h = ctypes.c_void_p()
    _check(lib().cos_build_propagators(ctypes.byref(m), _stream(stream), ctypes.byref(h)), "cos_build_propagators")
    return Tables(h)


def tables_for(model, stream=None) -> Tables:
    """Tables for an inputs.Model."""
    return cos_build_propagators(model.L, model.t, model.beta, model.U, model.mu, model.alpha, model.n_tau, stream)


def cos_build_propagators_honeycomb(L: int, t: float, beta: float, U: float, mu: Sequence[float],
                                    alpha: Sequence[float], delta: Sequence[float], n_tau: int,
                                    stream=None) -> Tables:
    nf = len(mu)
    arr = lambda v: (ctypes.c_double * nf)(*[float(x) for x in v])
    m = cos_honeycomb_model(int(L), float(t), float(beta), float(U), nf, arr(mu), arr(alpha), arr(delta), int(n_tau))
    h = ctypes.c_void_p()
    _check(lib().cos_build_propagators_honeycomb(ctypes.byref(m), _stream(stream), ctypes.byref(h)),
           "cos_build_propagators_honeycomb")
    return Tables(h)


def honeycomb_tables_for(model, stream=None) -> Tables:
    """Tables for an inputs.HoneycombModel."""
    return cos_build_propagators_honeycomb(model.L, model.t, model.beta, model.U, model.mu, model.alpha, model.delta,
                                           model.n_tau, stream)


def cos_gather_bipartite(tables: Tables, order, offset, site, tau, moff, M4, stream=None):
    _check(lib().cos_gather_bipartite(tables.handle, int(order.numel()), _ptr(order, "i32"), _ptr(offset, "i64"),
                                      _ptr(site, "i32"), _ptr(tau, "f64"), _ptr(moff, "i64"), _ptr(M4, "f64"),
                                      _stream(stream)), "cos_gather_bipartite")


def cos_bipartite_structure(n: int) -> cos_structure_info:
    inf = cos_structure_info()
    _check(lib().cos_bipartite_structure(int(n), ctypes.byref(inf)), "cos_bipartite_structure")
    return inf


def bipartite_matrix_offsets(order: np.ndarray, n_mat: int) -> np.ndarray:
    """Offsets of packed [n_mat][2 n_c][2 n_c] blocks for the given orders."""
    return matrix_offsets(2 * np.asarray(order, dtype=np.int64), n_mat)


def cos_gather(tables: Tables, order, offset, site, tau, moff, M, stream=None):
    _check(lib().cos_gather(tables.handle, int(order.numel()), _ptr(order, "i32"), _ptr(offset, "i64"), _ptr(site, "i32"), _ptr(tau, "f64"),
                            _ptr(moff, "i64"), _ptr(M, "f64"), _stream(stream)), "cos_gather")


def cos_connected_sum_matrices(n_max: int, order, moff, n_mat: int, loop_weight: int,
                               sigma: Optional[Sequence[float]], M, precision: str, out, abs_mass=None,
                               stream=None):
    sig = None
    if sigma is not None:
        sig = (ctypes.c_double * n_mat)(*[float(s) for s in sigma])
    _check(lib().cos_connected_sum_matrices(int(order.numel()), int(n_max), _ptr(order, "i32"), _ptr(moff, "i64"), int(n_mat),
                                            int(loop_weight), sig, _ptr(M, "f64"), PRECISIONS[precision], _ptr(out, "f64"),
                                            _ptr(abs_mass, "f64"), _stream(stream)), "cos_connected_sum_matrices")


def cos_connected_sum_matrices_noalloc(n_max: int, order, moff, n_mat: int, loop_weight: int,
                                       sigma: Optional[Sequence[float]], M, precision: str, out, abs_mass=None,
                                       stream=None):
    """cos_connected_sum_matrices without device allocation (fixed 128 MiB static workspace)."""
    sig = None
    if sigma is not None:
        sig = (ctypes.c_double * n_mat)(*[float(s) for s in sigma])
    _check(lib().cos_connected_sum_matrices_noalloc(int(order.numel()), int(n_max), _ptr(order, "i32"), _ptr(moff, "i64"),
                                                    int(n_mat), int(loop_weight), sig, _ptr(M, "f64"),
                                                    PRECISIONS[precision], _ptr(out, "f64"), _ptr(abs_mass, "f64"),
                                                    _stream(stream)), "cos_connected_sum_matrices_noalloc")


def cos_connected_sum_batch(tables: Tables, n_max: int, order, offset, site, tau, precision: str, out,
                            abs_mass=None, stream=None):
    _check(lib().cos_connected_sum_batch(tables.handle, int(order.numel()), int(n_max), _ptr(order, "i32"), _ptr(offset, "i64"),
                                         _ptr(site, "i32"), _ptr(tau, "f64"), PRECISIONS[precision], _ptr(out, "f64"), _ptr(abs_mass, "f64"),
                                         _stream(stream)), "cos_connected_sum_batch")


def cos_connected_sum_grad(tables: Tables, n_max: int, order, offset, site, tau, gout, out=None, gM=None,
                           gmoff=None, gmu=None, galpha=None, stream=None):
    _check(lib().cos_connected_sum_grad(tables.handle, int(order.numel()), int(n_max), _ptr(order, "i32"), _ptr(offset, "i64"),
                                        _ptr(site, "i32"), _ptr(tau, "f64"), _ptr(gout, "f64"), _ptr(out, "f64"), _ptr(gM, "f64"), _ptr(gmoff, "i64"),
                                        _ptr(gmu, "f64"), _ptr(galpha, "f64"), _stream(stream)), "cos_connected_sum_grad")


# ------------------------------------------------------------------ cos_problem (one call per operation)

def _shifts(shift, count: int):
    """Host shift weights as a C array of `count` doubles (or NULL)."""
    if shift is None:
        return None
    flat = [float(x) for x in np.asarray(shift, dtype=np.float64).ravel()]
    if len(flat) != count:
        raise ValueError(f"expected {count} shift weights, got {len(flat)}")
    return (ctypes.c_double * count)(*flat)


def problem(lattice: int, weights: int, precision: str, n_max: int, order, tables: Optional["Tables"] = None,
            offset=None, site=None, tau=None, moff=None, M=None, n_mat: int = 0, loop_weight: int = 0,
            shift=None) -> cos_problem:
    """A cos_problem for cos_forward / cos_grad / cos_subsets: vertex coordinates (tables,
    offset, site, tau) or explicit matrices (moff, M, n_mat, loop_weight); `shift` as the
    weight kind expects (square loops [n_mat], bipartite loops [n_mat][2], determinant weights
    [2] or [2][2])."""
    p = cos_problem()
    p.lattice, p.weights, p.precision = int(lattice), int(weights), PRECISIONS[precision]
    p.n_cfg, p.n_max = int(order.numel()), int(n_max)
    p.d_order = _ptr(order, "i32").value
    h = tables.handle if tables is not None else None
    p.tables = h.value if isinstance(h, ctypes.c_void_p) else h
    p.d_offset = _ptr(offset, "i64").value
    p.d_site = _ptr(site, "i32").value
    p.d_tau = _ptr(tau, "f64").value
    p.d_moff = _ptr(moff, "i64").value
    p.d_M = _ptr(M, "f64").value
    p.n_mat, p.loop_weight = int(n_mat), int(loop_weight)
    if shift is not None:
        count = (2 if weights == COS_DETERMINANTS else int(n_mat)) * (2 if lattice == COS_BIPARTITE else 1)
        arr = _shifts(shift, count)
        p.h_shift = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
        p._keep = arr   # the array lives as long as the descriptor
    return p


def cos_forward(p: cos_problem, out, abs_mass=None, stream=None):
    _check(lib().cos_forward(ctypes.byref(p), _ptr(out, "f64"), _ptr(abs_mass, "f64"), _stream(stream)), "cos_forward")


def cos_grad(p: cos_problem, gout, out=None, gM=None, gmoff=None, gshift=None, gmu=None, galpha=None, stream=None):
    _check(lib().cos_grad(ctypes.byref(p), _ptr(gout, "f64"), _ptr(out, "f64"), _ptr(gM, "f64"), _ptr(gmoff, "i64"),
                          _ptr(gshift, "f64"), _ptr(gmu, "f64"), _ptr(galpha, "f64"), _stream(stream)), "cos_grad")


def cos_subsets(p: cos_problem, c_out, a_out=None, all_roots: bool = True, stream=None):
    _check(lib().cos_subsets(ctypes.byref(p), int(bool(all_roots)), _ptr(c_out, "f64"), _ptr(a_out, "f64"),
                             _stream(stream)), "cos_subsets")


# The per-case calls of earlier versions, kept as Python functions over the descriptor calls.

def cos_connected_sum_matrices_grad(n_max: int, order, moff, n_mat: int, loop_weight: int,
                                    sigma: Optional[Sequence[float]], M, gout, out=None, gM=None, gsigma=None,
                                    stream=None):
    """Gradient of the connected sums of explicit matrices: dLoss/dM (layout of M) and
    dLoss/dsigma ([n_cfg][n_mat]) for dLoss/dc = gout."""
    cos_grad(problem(COS_SQUARE, COS_LOOPS, "fp64", n_max, order, moff=moff, M=M, n_mat=n_mat,
                     loop_weight=loop_weight, shift=sigma), gout, out, gM, gshift=gsigma, stream=stream)


def cos_connected_sum_subsets(n_max: int, order, moff, n_mat: int, loop_weight: int,
                              sigma: Optional[Sequence[float]], M, precision: str, c_out, a_out=None,
                              all_roots: bool = True, stream=None):
    """c(S) (and a(S) when a_out is given) of every vertex subset S: c_out / a_out are
    [n_cfg * 2^n_max] float64, entry c * 2^n_max + S (bit i of S = vertex i)."""
    cos_subsets(problem(COS_SQUARE, COS_LOOPS, precision, n_max, order, moff=moff, M=M, n_mat=n_mat,
                        loop_weight=loop_weight, shift=sigma), c_out, a_out, all_roots, stream)


def cos_connected_sum_bipartite_matrices(n_max: int, order, moff, n_mat: int, loop_weight: int, sigma2, M4,
                                         precision: str, out, abs_mass=None, stream=None):
    """Bipartite connected sums of explicit matrices; sigma2: None or n_mat x 2 shift weights
    (flavor, sublattice)."""
    cos_forward(problem(COS_BIPARTITE, COS_LOOPS, precision, n_max, order, moff=moff, M=M4, n_mat=n_mat,
                        loop_weight=loop_weight, shift=sigma2), out, abs_mass, stream)


def cos_connected_sum_bipartite_batch(tables: "Tables", n_max: int, order, offset, site, tau, precision: str, out,
                                      abs_mass=None, stream=None):
    cos_forward(problem(COS_BIPARTITE, COS_LOOPS, precision, n_max, order, tables, offset, site, tau), out,
                abs_mass, stream)


def cos_connected_sum_bipartite_matrices_grad(n_max: int, order, moff, n_mat: int, loop_weight: int, sigma2, M4,
                                              gout, out=None, gM4=None, gsigma2=None, stream=None):
    """Gradient of the bipartite sums: dLoss/dM4 (layout of M4) and dLoss/dsigma2 ([n_cfg][n_mat][2])."""
    cos_grad(problem(COS_BIPARTITE, COS_LOOPS, "fp64", n_max, order, moff=moff, M=M4, n_mat=n_mat,
                     loop_weight=loop_weight, shift=sigma2), gout, out, gM4, gshift=gsigma2, stream=stream)


def cos_connected_sum_bipartite_grad(tables: "Tables", n_max: int, order, offset, site, tau, gout, out=None, gM4=None,
                                     gmoff=None, gmu=None, galpha=None, stream=None):
    """Gradient of the bipartite sums from vertex coordinates (honeycomb tables): dLoss/dM4
    ([n_mat][2 n_c][2 n_c] at gmoff), dLoss/dmu and dLoss/dalpha ([n_cfg][n_flavors])."""
    cos_grad(problem(COS_BIPARTITE, COS_LOOPS, "fp64", n_max, order, tables, offset, site, tau), gout, out, gM4,
             gmoff, None, gmu, galpha, stream)


def cos_connected_sum_bipartite_subsets(n_max: int, order, moff, n_mat: int, loop_weight: int, sigma2, M4, c_out,
                                        a_out=None, all_roots: bool = True, stream=None):
    """c(S) (and a(S)) of every vertex subset S on a bipartite lattice."""
    cos_subsets(problem(COS_BIPARTITE, COS_LOOPS, "fp64", n_max, order, moff=moff, M=M4, n_mat=n_mat,
                        loop_weight=loop_weight, shift=sigma2), c_out, a_out, all_roots, stream)


def cos_connected_det_matrices(n_max: int, order, moff, alpha: Optional[Sequence[float]], M, precision: str, out,
                               abs_mass=None, stream=None):
    """SU(2) determinant weights (Alg. 1): M holds [2][n_c][n_c] (spin up, spin down) per
    configuration at moff; alpha None or the two diagonal shifts."""
    cos_forward(problem(COS_SQUARE, COS_DETERMINANTS, precision, n_max, order, moff=moff, M=M, shift=alpha), out,
                abs_mass, stream)


def cos_connected_det_batch(tables: "Tables", n_max: int, order, offset, site, tau, alpha, precision: str, out,
                            abs_mass=None, stream=None):
    """Gather + SU(2) determinant-weight sums from vertex coordinates (SU(2) tables built with
    alpha = 0; alpha: None or the two diagonal shifts)."""
    cos_forward(problem(COS_SQUARE, COS_DETERMINANTS, precision, n_max, order, tables, offset, site, tau,
                        shift=alpha), out, abs_mass, stream)


def cos_connected_det_matrices_grad(n_max: int, order, moff, alpha: Optional[Sequence[float]], M, gout, out=None,
                                    gM=None, galpha=None, stream=None):
    """Gradient of the SU(2) determinant-weight sums: dLoss/dM (layout of M) and dLoss/dalpha
    ([n_cfg][2]) for dLoss/dc = gout."""
    cos_grad(problem(COS_SQUARE, COS_DETERMINANTS, "fp64", n_max, order, moff=moff, M=M, shift=alpha), gout, out,
             gM, gshift=galpha, stream=stream)


def cos_connected_det_grad(tables: "Tables", n_max: int, order, offset, site, tau, alpha, gout, out=None, gM=None,
                           gmoff=None, gmu=None, galpha=None, stream=None):
    """Gradient of the SU(2) determinant-weight sums from vertex coordinates: dLoss/dM ([2][n_c][n_c]
    at gmoff), dLoss/dmu and dLoss/dalpha ([n_cfg][2], alpha the diagonal shifts)."""
    cos_grad(problem(COS_SQUARE, COS_DETERMINANTS, "fp64", n_max, order, tables, offset, site, tau, shift=alpha),
             gout, out, gM, gmoff, galpha, gmu, None, stream)


def cos_connected_det_subsets(n_max: int, order, moff, alpha: Optional[Sequence[float]], M, c_out, a_out=None,
                              all_roots: bool = True, stream=None):
    """c(S) (and a(S) = det(A_up[S]) det(A_dn[S]) when a_out is given) of every vertex subset S
    for determinant weights."""
    cos_subsets(problem(COS_SQUARE, COS_DETERMINANTS, "fp64", n_max, order, moff=moff, M=M, shift=alpha), c_out,
                a_out, all_roots, stream)


def cos_connected_det_bipartite_matrices(n_max: int, order, moff, alpha2, M4, precision: str, out, abs_mass=None,
                                         stream=None):
    """SU(2) determinant weights on a bipartite lattice (Alg. 1): M4 holds [2][2 n_c][2 n_c]
    per configuration at moff; alpha2 None or 2 x 2 diagonal shifts (spin, sublattice)."""
    cos_forward(problem(COS_BIPARTITE, COS_DETERMINANTS, precision, n_max, order, moff=moff, M=M4, shift=alpha2),
                out, abs_mass, stream)


def cos_connected_det_bipartite_batch(tables: "Tables", n_max: int, order, offset, site, tau, alpha2, precision: str,
                                      out, abs_mass=None, stream=None):
    """Gather + bipartite determinant-weight sums from vertex coordinates (two-flavor honeycomb
    tables; alpha2: None or the 2 x 2 diagonal shifts, spin then sublattice)."""
    cos_forward(problem(COS_BIPARTITE, COS_DETERMINANTS, precision, n_max, order, tables, offset, site, tau,
                        shift=alpha2), out, abs_mass, stream)


def cos_connected_det_bipartite_matrices_grad(n_max: int, order, moff, alpha2, M4, gout, out=None, gM4=None,
                                              galpha2=None, stream=None):
    """Gradient of the bipartite determinant-weight sums: dLoss/dM4 and dLoss/dalpha2 ([n_cfg][2][2])."""
    cos_grad(problem(COS_BIPARTITE, COS_DETERMINANTS, "fp64", n_max, order, moff=moff, M=M4, shift=alpha2), gout,
             out, gM4, gshift=galpha2, stream=stream)


def cos_connected_det_bipartite_grad(tables: "Tables", n_max: int, order, offset, site, tau, alpha2, gout, out=None,
                                     gM4=None, gmoff=None, gmu=None, galpha2=None, stream=None):
    """Gradient of the bipartite determinant-weight sums from vertex coordinates: dLoss/dM4
    ([2][2 n_c][2 n_c] at gmoff), dLoss/dmu ([n_cfg][2]) and dLoss/dalpha2 ([n_cfg][2][2])."""
    cos_grad(problem(COS_BIPARTITE, COS_DETERMINANTS, "fp64", n_max, order, tables, offset, site, tau, shift=alpha2),
             gout, out, gM4, gmoff, galpha2, gmu, None, stream)


def cos_connected_det_bipartite_subsets(n_max: int, order, moff, alpha2, M4, c_out, a_out=None,
                                        all_roots: bool = True, stream=None):
    """c(S) (and a(S)) of every vertex subset S for bipartite determinant weights."""
    cos_subsets(problem(COS_BIPARTITE, COS_DETERMINANTS, "fp64", n_max, order, moff=moff, M=M4, shift=alpha2),
                c_out, a_out, all_roots, stream)


def cos_sync_status(stream=None):
    _check(lib().cos_sync_status(_stream(stream)), "cos_sync_status")


def cos_release_workspace(stream=None):
    """Free the library's device workspace of this stream (after reporting its status)."""
    _check(lib().cos_release_workspace(_stream(stream)), "cos_release_workspace")


def cos_structure(n: int) -> cos_structure_info:
    inf = cos_structure_info()
    _check(lib().cos_structure(int(n), ctypes.byref(inf)), "cos_structure")
    return inf


def cos_grad_checkpoint_plan(n: int, slots_budget: int = 0):
    """(checkpoint layer mask, slots per lane kept, multiply-adds re-run) of the gradient's
    plan at order n for a budget of state slots per lane (0: the least storage)."""
    m, st, rc = ctypes.c_uint32(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().cos_grad_checkpoint_plan(int(n), int(slots_budget), ctypes.byref(m), ctypes.byref(st),
                                          ctypes.byref(rc)), "cos_grad_checkpoint_plan")
    return m.value, st.value, rc.value


# ------------------------------------------------------------------ torch-facing helpers

def configs_to_device(cfgs, device="cuda"):
    """Device copies (order int32, offset int64, site int32, tau float64) of inputs.Configs."""
    import torch
    return (torch.as_tensor(cfgs.order, dtype=torch.int32, device=device),
            torch.as_tensor(cfgs.offset, dtype=torch.int64, device=device),
            torch.as_tensor(cfgs.site, dtype=torch.int32, device=device),
            torch.as_tensor(cfgs.tau, dtype=torch.float64, device=device))


def matrix_offsets(order: np.ndarray, n_mat: int) -> np.ndarray:
    """Offsets of packed [n_mat][n_c][n_c] blocks for the given orders."""
    sizes = n_mat * np.asarray(order, dtype=np.int64) ** 2
    off = np.zeros(len(sizes), dtype=np.int64)
    if len(sizes):
        off[1:] = np.cumsum(sizes[:-1])
    return off


_instr = None


def instr_lib():
    """The benchmark's and tests' instruments (FMA probe, scattered-row traffic, conversion check), built beside
    libcos.so into libcos_instr.so; not part of the library's interface."""
    global _instr
    if _instr is None:
        lib()   # builds both libraries when sources changed
        L = ctypes.CDLL(os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcos_instr.so"))
        vp = ctypes.c_void_p
        L.cos_instr_fma_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
        L.cos_instr_fma_probe.restype = ctypes.c_int
        L.cos_instr_convert_check.argtypes = [ctypes.c_int64, vp, vp, vp, vp, vp]
        L.cos_instr_convert_check.restype = ctypes.c_int
        L.cos_instr_row_traffic.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp,
                                            ctypes.c_int64, vp]
        L.cos_instr_row_traffic.restype = ctypes.c_int
        _instr = L
    return _instr


def _instr_check(rc: int, where: str):
    if rc != 0:
        raise RuntimeError(f"{where}: {'bad argument' if rc < 0 else 'CUDA error %d' % rc}")


def fma_probe(kind: int, blocks: int, threads: int, iters: int, sink, stream=None):
    _instr_check(instr_lib().cos_instr_fma_probe(int(kind), int(blocks), int(threads), int(iters), _ptr(sink),
                                                 _stream(stream)), "cos_instr_fma_probe")


def row_traffic(mode: int, ilp: int, blocks: int, threads: int, iters: int, src, dst, stream=None):
    """Scattered 512-byte rows (mode 0 read + write, 1 read, 2 write) over src / dst (equal
    byte sizes, a multiple of 512)."""
    nrows = min(src.numel() * src.element_size(), dst.numel() * dst.element_size()) // 512
    _instr_check(instr_lib().cos_instr_row_traffic(int(mode), int(ilp), int(blocks), int(threads), int(iters),
                                                   _ptr(src), _ptr(dst), int(nrows), _stream(stream)),
                 "cos_instr_row_traffic")


def probe_sweep(gib: int = 4):
    """Issue-side rates of this GPU, for the design of the DP kernels: the FP64 FMA rate by
    independent chains per thread and warps per SM (one CTA per SM), and the DRAM rate of
    scattered 512-byte row traffic by warps per SM and rows in flight per warp (two buffers of
    `gib` GiB).  Returns a list of result dicts."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    clock = 2.032e9
    out = []

    def best_ms(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    for kind, chains in ((5, 1), (6, 2), (2, 4), (0, 8), (3, 16)):
        for threads in (32, 64, 96, 128, 256, 512):
            sink = torch.zeros(sms, dtype=torch.float64, device="cuda")
            it = 4096
            ms = best_ms(lambda: fma_probe(kind, sms, threads, it, sink))
            tf = 2.0 * sms * threads * chains * it / (ms * 1e-3) / 1e12
            out.append({"probe": "fp64_fma", "chains_per_thread": chains, "warps_per_sm": threads // 32,
                        "tflops": tf, "lanes_per_clk_per_sm_at_2032mhz": tf * 1e12 / 2 / sms / clock})
    nbytes = gib << 30
    a = torch.zeros(nbytes // 4, dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    iters = 64
    for threads in (256, 512, 1024):
        for ilp in (1, 4, 8):
            ms = best_ms(lambda: row_traffic(0, ilp, sms, threads, iters, a, b))
            moved = sms * threads / 32 * iters * ilp * 512 * 2
            out.append({"probe": "row_traffic_read_write", "warps_per_sm": threads // 32, "rows_in_flight": ilp,
                        "gb_per_s": moved / (ms * 1e-3) / 1e9})
    for mode, name in ((1, "row_traffic_read"), (2, "row_traffic_write")):
        ms = best_ms(lambda: row_traffic(mode, 8, sms, 1024, iters, a, b))
        moved = sms * 1024 / 32 * iters * 8 * 512
        out.append({"probe": name, "warps_per_sm": 32, "rows_in_flight": 8, "gb_per_s": moved / (ms * 1e-3) / 1e9})
    del a, b
    return out


def convert_check(in64, in32, narrowed, widened, stream=None):
    _instr_check(instr_lib().cos_instr_convert_check(int(in64.numel()), _ptr(in64, "f64"), _ptr(in32),
                                                     _ptr(narrowed), _ptr(widened, "f64"), _stream(stream)),
                 "cos_instr_convert_check")


def measure_peak(kind: int = 0, iters: int = 4096, reps: int = 3, sweep: bool = False):
    """Measured FMA throughput (FLOP/s) of the FP64 (kind 0) or FP32 (kind 1) pipe: the best
    of `reps` launches; with sweep=True (FP64) the best over chains per thread {4, 8, 16, 32}
    and block shapes, returned with the shape that reached it."""
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    chains_of = {0: 8, 1: 16, 2: 4, 3: 16, 4: 32, 5: 1, 6: 2}
    shapes = [(kind, 256, 8)]
    if sweep and kind == 0:
        shapes = [(k, t, b) for k in (2, 0, 3, 4) for t in (128, 256, 512) for b in (1, 2, 4, 8) if t * b <= 2048]
    best, best_shape = 0.0, None
    for k, threads, per_sm in shapes:
        blocks = sms * per_sm
        chains = chains_of[k]
        sink = torch.zeros(blocks, dtype=torch.float64 if k != 1 else torch.float32, device="cuda")
        it = max(64, iters * 8 // chains)
        fma_probe(k, blocks, threads, 64, sink)                    # warm-up
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            fma_probe(k, blocks, threads, it, sink)
            e1.record()
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3
            rate = 2.0 * blocks * threads * chains * it / sec
            if rate > best:
                best, best_shape = rate, {"chains": chains, "threads": threads, "ctas_per_sm": per_sm}
    return (best, best_shape) if sweep else best


class Plan:
    """A batch frozen into a CUDA graph (cos_plan_*); keep the tensors it references alive."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def launch(self, stream=None):
        _check(lib().cos_plan_launch(self.handle, _stream(stream)), "cos_plan_launch")

    def status(self, stream=None):
        _check(lib().cos_plan_status(self.handle, _stream(stream)), "cos_plan_status")

    def grid(self) -> int:
        g = ctypes.c_int()
        _check(lib().cos_plan_grid(self.handle, ctypes.byref(g)), "cos_plan_grid")
        return g.value

    def close(self):
        if self.handle:
            lib().cos_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cos_plan_create_batch(tables: Tables, n_max: int, order, offset, site, tau, precision: str, out, abs_mass=None,
                          stream=None) -> Plan:
    h = ctypes.c_void_p()
    _check(lib().cos_plan_create_batch(tables.handle, int(order.numel()), int(n_max), _ptr(order, "i32"),
                                       _ptr(offset, "i64"), _ptr(site, "i32"), _ptr(tau, "f64"),
                                       PRECISIONS[precision], _ptr(out, "f64"), _ptr(abs_mass, "f64"),
                                       _stream(stream), ctypes.byref(h)), "cos_plan_create_batch")
    return Plan(h, (tables, order, offset, site, tau, out, abs_mass))


def cos_plan_create_matrices(n_max: int, order, moff, n_mat: int, loop_weight: int, sigma, M, precision: str, out,
                             abs_mass=None, stream=None) -> Plan:
    sig = None
    if sigma is not None:
        sig = (ctypes.c_double * n_mat)(*[float(s) for s in sigma])
    h = ctypes.c_void_p()
    _check(lib().cos_plan_create_matrices(int(order.numel()), int(n_max), _ptr(order, "i32"), _ptr(moff, "i64"),
                                          int(n_mat), int(loop_weight), sig, _ptr(M, "f64"), PRECISIONS[precision],
                                          _ptr(out, "f64"), _ptr(abs_mass, "f64"), _stream(stream), ctypes.byref(h)),
           "cos_plan_create_matrices")
    return Plan(h, (order, moff, M, out, abs_mass))


def cos_set_tuning(n: int, precision: str, n_mat: int, warps: int, ctas_per_sm: int, prefetch: int = 1):
    _check(lib().cos_set_tuning(n, PRECISIONS[precision], n_mat, warps, ctas_per_sm, int(prefetch)),
           "cos_set_tuning")


def cos_get_tuning(n: int, precision: str, n_mat: int):
    """(warps per CTA, CTAs per SM, prefetch) of the DP launch for this case."""
    w, c, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().cos_get_tuning(n, PRECISIONS[precision], n_mat, ctypes.byref(w), ctypes.byref(c), ctypes.byref(p)),
           "cos_get_tuning")
    return w.value, c.value, p.value


def cos_autotune(n: int, n_mat: int, loop_weight: int, shifts: bool, precision: str, n_cfg: int, stream=None):
    """Times the DP launch shapes for order n and installs the fastest; returns (warps, ctas, prefetch, ms)."""
    w, c, p, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().cos_autotune(n, n_mat, loop_weight, int(shifts), PRECISIONS[precision], n_cfg, _stream(stream),
                              ctypes.byref(w), ctypes.byref(c), ctypes.byref(p), ctypes.byref(ms)), "cos_autotune")
    return w.value, c.value, p.value, ms.value
