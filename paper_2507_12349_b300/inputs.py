"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module holds no arithmetic of the method itself: only the counter-based
random generator that draws Monte Carlo configurations (vertex sites and
imaginary times) and the parameter sets of the benchmark workloads.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  Each uniform is the SplitMix64 output for a
counter built from (seed, configuration, vertex, field), so any single value
can be regenerated on its own.  A 53-bit uniform u in [0, 1) gives
site = floor(u * L^2) (site = x + L*y) and tau = u * beta.  Orders of the
uneven workload are n = n_lo + floor(u * (n_hi - n_lo + 1)).

The workloads restate the five benchmark configurations: square-lattice SU(N)
Hubbard models (Methods A of the paper) at the orders the paper's physics runs
reach (up to 8-9, Results B) and beyond, with sites uniform on an L x L torus
and times uniform in [0, beta).  They stand in for the Monte Carlo samples of
the paper's 32 x 32 runs; no dataset exists to fetch.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

FIELD_SITE = 0
FIELD_TAU = 1
FIELD_ORDER = 2
VERTEX_PER_CONFIG = 255  # vertex slot used for per-configuration draws


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output for state `counter` (uint64 array, wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = np.asarray(counter, dtype=np.uint64) + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def counter(seed: int, cfg: np.ndarray, vertex: np.ndarray, fld: int) -> np.ndarray:
    """Counter seed*2^32 + cfg*2^10 + vertex*4 + field (cfg < 2^22, vertex < 256, field < 4)."""
    cfg = np.asarray(cfg, dtype=np.uint64)
    vertex = np.asarray(vertex, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return ((np.uint64(seed) << np.uint64(32)) + (cfg << np.uint64(10))
                + (vertex << np.uint64(2)) + np.uint64(fld))


def uniform53(seed: int, cfg, vertex, fld: int) -> np.ndarray:
    """53-bit uniform in [0, 1) for each (cfg, vertex) pair."""
    z = splitmix64(counter(seed, cfg, vertex, fld))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass(frozen=True)
class Model:
    """Square-lattice SU(N_f) Hubbard model (Methods A): hopping t, inverse
    temperature beta, interaction U, per-flavor chemical potential mu and shift
    alpha, L x L periodic lattice, n_tau imaginary-time grid points."""
    L: int
    t: float
    beta: float
    U: float
    mu: tuple
    alpha: tuple
    n_tau: int

    @property
    def n_flavors(self) -> int:
        return len(self.mu)

    @property
    def symmetric(self) -> bool:
        """All flavors share one propagator and one shift: SU(N) symmetric."""
        return len(set(self.mu)) == 1 and len(set(self.alpha)) == 1

    @property
    def sigma(self) -> tuple:
        """Shift weights sigma_lambda = alpha_lambda / U (equal-time shift, Methods A)."""
        return tuple(a / self.U for a in self.alpha)


@dataclass(frozen=True)
class HoneycombModel:
    """Honeycomb-lattice SU(N_f) Hubbard model (Methods A, bipartite lattices): L x L unit
    cells of two sites (sublattices A, B), hopping t, inverse temperature beta, interaction U,
    per-flavor chemical potential mu, uniform shift alpha and staggered shift delta (+delta
    on A, -delta on B), n_tau imaginary-time grid points.  A vertex sits in a unit cell
    (site = r_1 + L r_2 in cell coordinates along the two lattice vectors); its sublattice is
    summed over."""
    L: int
    t: float
    beta: float
    U: float
    mu: tuple
    alpha: tuple
    delta: tuple
    n_tau: int

    @property
    def n_flavors(self) -> int:
        return len(self.mu)

    @property
    def symmetric(self) -> bool:
        return len(set(self.mu)) == 1 and len(set(self.alpha)) == 1 and len(set(self.delta)) == 1

    @property
    def sigma2(self) -> tuple:
        """Shift weights per (flavor, sublattice): (alpha + delta) / U on A, (alpha - delta) / U
        on B (the sublattice-dependent equal-time shift of Methods A)."""
        return tuple(((a + d) / self.U, (a - d) / self.U) for a, d in zip(self.alpha, self.delta))


@dataclass(frozen=True)
class Workload:
    name: str
    model: Model
    n_lo: int
    n_hi: int
    n_cfg: int
    seed: int
    precision: str  # "fp64" or "mixed"
    grad: bool = False
    det: bool = False   # SU(2) determinant weights (spin blocks up, down; no cycle factors)


WORKLOADS = {
    "su2_sym_n4": Workload("su2_sym_n4", Model(8, 1.0, 2.0, 2.0, (0.0, 0.0), (0.0, 0.0), 512),
                           4, 4, 10_000, 0, "fp64"),
    "su4_mu_broken_n8": Workload("su4_mu_broken_n8",
                                 Model(16, 1.0, 4.0, 1.5, (-0.3, -0.1, 0.1, 0.3), (0.0,) * 4, 1024),
                                 8, 8, 100_000, 1, "fp64"),
    "su3_shift_mixed_n10": Workload("su3_shift_mixed_n10",
                                    Model(16, 1.0, 4.0, 2.0, (0.0,) * 3, (0.2, 0.0, -0.2), 1024),
                                    10, 10, 100_000, 2, "mixed"),
    "su6_sym_uneven_n4_12": Workload("su6_sym_uneven_n4_12",
                                     Model(32, 1.0, 6.0, 1.0, (0.1,) * 6, (0.0,) * 6, 1024),
                                     4, 12, 200_000, 3, "fp64"),
    "su4_adjoint_n10": Workload("su4_adjoint_n10",
                                Model(16, 1.0, 4.0, 1.5, (-0.2, 0.0, 0.0, 0.2), (0.0,) * 4, 1024),
                                10, 10, 50_000, 4, "fp64", grad=True),
    # Honeycomb (two sublattices, summed per vertex): SU(2) with an antiferromagnetic
    # staggered shift (delta of opposite sign for the two spins), half filling, the paper's
    # honeycomb physics orders (up to 8).
    "hc_su2_af_n8": Workload("hc_su2_af_n8",
                             HoneycombModel(16, 1.0, 6.0, 3.0, (0.0, 0.0), (0.0, 0.0), (0.25, -0.25), 1024),
                             8, 8, 20_000, 5, "fp64"),
    # SU(2) on the square lattice with determinant weights n_up n_dn and a Zeeman split of the
    # chemical potential (spin-dependent mu, so the two spin blocks differ), order 10.
    "su2_zeeman_det_n10": Workload("su2_zeeman_det_n10",
                                   Model(16, 1.0, 4.0, 2.0, (-0.2, 0.2), (0.0, 0.0), 1024),
                                   10, 10, 20_000, 6, "fp64", det=True),
}


@dataclass
class Configs:
    """A batch of configurations packed by configuration (uneven orders allowed).

    order[c]  : number of vertices n_c of configuration c
    offset[c] : start of configuration c in `site` / `tau`
    site[k]   : lattice site x + L*y of vertex k, in [0, L^2)
    tau[k]    : imaginary time of vertex k, in [0, beta)
    """
    order: np.ndarray
    offset: np.ndarray
    site: np.ndarray
    tau: np.ndarray

    @property
    def n_cfg(self) -> int:
        return int(self.order.shape[0])

    def subset(self, idx: Sequence[int]) -> "Configs":
        idx = np.asarray(idx, dtype=np.int64)
        order = self.order[idx].astype(np.int32)
        offset = np.zeros(len(idx), dtype=np.int64)
        if len(idx):
            offset[1:] = np.cumsum(order[:-1].astype(np.int64))
        pos = np.concatenate([np.arange(self.offset[i], self.offset[i] + self.order[i]) for i in idx]) \
            if len(idx) else np.zeros(0, dtype=np.int64)
        return Configs(order, offset, self.site[pos].astype(np.int32), self.tau[pos].astype(np.float64))


def make_configs(model, n_lo: int, n_hi: int, n_cfg: int, seed: int,
                 first_cfg: int = 0) -> Configs:
    """Configurations first_cfg .. first_cfg+n_cfg-1 of the seeded stream."""
    cfg = np.arange(first_cfg, first_cfg + n_cfg, dtype=np.uint64)
    if n_lo == n_hi:
        order = np.full(n_cfg, n_lo, dtype=np.int32)
    else:
        u = uniform53(seed, cfg, np.full(n_cfg, VERTEX_PER_CONFIG, dtype=np.uint64), FIELD_ORDER)
        order = (n_lo + np.floor(u * (n_hi - n_lo + 1))).astype(np.int32)
        order = np.minimum(order, n_hi)
    offset = np.zeros(n_cfg, dtype=np.int64)
    if n_cfg:
        offset[1:] = np.cumsum(order[:-1].astype(np.int64))
    total = int(order.sum())
    cfg_of = np.repeat(cfg, order.astype(np.int64))
    vtx = (np.arange(total, dtype=np.int64) - np.repeat(offset, order.astype(np.int64))).astype(np.uint64)
    L2 = model.L * model.L
    us = uniform53(seed, cfg_of, vtx, FIELD_SITE)
    ut = uniform53(seed, cfg_of, vtx, FIELD_TAU)
    site = np.minimum(np.floor(us * L2), L2 - 1).astype(np.int32)
    tau = ut * model.beta
    return Configs(order, offset, site, tau)


def workload_configs(w: Workload, n_cfg: Optional[int] = None, first_cfg: int = 0) -> Configs:
    return make_configs(w.model, w.n_lo, w.n_hi, w.n_cfg if n_cfg is None else n_cfg, w.seed, first_cfg)


def random_matrices(seed: int, n_cfg: int, n_flavors: int, n: int, scale: float = 1.0) -> np.ndarray:
    """Dense random test matrices [cfg][flavor][n][n], entries uniform in [-scale, scale)."""
    cfg = np.repeat(np.arange(n_cfg, dtype=np.uint64), n_flavors * n * n)
    k = np.tile(np.arange(n_flavors * n * n, dtype=np.uint64), n_cfg)
    z = splitmix64((np.uint64(seed) << np.uint64(40)) + (cfg << np.uint64(16)) + k)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (scale * (2.0 * u - 1.0)).reshape(n_cfg, n_flavors, n, n)
