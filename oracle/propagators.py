"""Free propagator tables and the gather into per-configuration matrices.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Methods A, square lattice: the flavor-l dispersion is
    xi_l(k) = -2t [cos k_x + cos k_y] - mu_l + alpha_l,   k = 2 pi (m_x, m_y) / L,
and the imaginary-time propagator, with G0(r, tau) = -<T c(r, tau) c^+(0, 0)>, is
    G0_l(r, tau) = -(1/L^2) sum_k cos(k.r) exp(-xi tau) (1 - n_F(xi)),  0 < tau < beta,
    G0_l(r, tau - beta) = -G0_l(r, tau)                                   (antiperiodic),
so that G0_l(r, 0^-) = (1/L^2) sum_k cos(k.r) n_F(xi) (the equal-time value, Methods A).

Readings (the paper does not state the grid): the table holds n_tau points
tau_m = m beta / (n_tau - 1), m = 0..n_tau-1, with G(0^+) at m = 0 and
G(beta^-) at the last point; entries between points are linear
interpolations; a time difference dt <= 0 (including dt = 0 and the diagonal
i = j) uses -G(dt + beta), i.e. equal times are taken at 0^-.

Every sum here is the plain definition: a dense cos(k.r) matrix times the
weight matrix over k (a library matmul), no symmetry reduction.
"""
from __future__ import annotations

import numpy as np


def fermi(x: np.ndarray, beta: float) -> np.ndarray:
    """n_F(x) = 1 / (exp(beta x) + 1), evaluated on the side where the
    exponential cannot overflow."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    pos = x >= 0
    e = np.exp(-beta * x[pos])
    out[pos] = e / (1.0 + e)
    out[~pos] = 1.0 / (1.0 + np.exp(beta * x[~pos]))
    return out


def tau_weight(x: np.ndarray, tau: np.ndarray, beta: float) -> np.ndarray:
    """w(x, tau) = exp(-x tau) (1 - n_F(x)) for 0 <= tau <= beta, outer product
    over (x, tau), in the two overflow-free forms
      x >= 0 : exp(-x tau) / (1 + exp(-beta x))
      x <  0 : exp(x (beta - tau)) / (1 + exp(beta x))."""
    x = np.asarray(x, dtype=np.float64)[:, None]
    tau = np.asarray(tau, dtype=np.float64)[None, :]
    pos = x >= 0
    a = np.exp(-np.where(pos, x, 0.0) * tau) / (1.0 + np.exp(-beta * np.where(pos, x, 0.0)))
    b = np.exp(np.where(pos, 0.0, x) * (beta - tau)) / (1.0 + np.exp(beta * np.where(pos, 0.0, x)))
    return np.where(pos, a, b)


def momenta(L: int):
    m = np.arange(L)
    kx, ky = np.meshgrid(2 * np.pi * m / L, 2 * np.pi * m / L, indexing="xy")
    return kx.ravel(), ky.ravel()   # index k = m_x + L m_y


def dispersion(L: int, t: float, mu: float, alpha: float) -> np.ndarray:
    kx, ky = momenta(L)
    return -2.0 * t * (np.cos(kx) + np.cos(ky)) - mu + alpha


def cos_kr(L: int) -> np.ndarray:
    """cos(k.r) for r = x + L y (rows) and k = m_x + L m_y (columns)."""
    kx, ky = momenta(L)
    r = np.arange(L * L)
    x, y = r % L, r // L
    return np.cos(np.outer(x, kx) + np.outer(y, ky))


def tau_grid(beta: float, n_tau: int) -> np.ndarray:
    return np.arange(n_tau) * beta / (n_tau - 1)


def table(L: int, t: float, beta: float, mu: float, alpha: float, n_tau: int) -> np.ndarray:
    """G0(r, tau_m) for 0^+ <= tau_m <= beta^-, shape [L^2][n_tau]."""
    xi = dispersion(L, t, mu, alpha)
    w = tau_weight(xi, tau_grid(beta, n_tau), beta)
    return -(cos_kr(L) @ w) / (L * L)


def dtable_dmu(L: int, t: float, beta: float, mu: float, alpha: float, n_tau: int) -> np.ndarray:
    """d G0(r, tau_m) / d mu.  With d xi / d mu = -1 and
    d/dxi [exp(-xi tau)(1 - n_F)] = exp(-xi tau)(1 - n_F)(-tau + beta n_F):
      dG/dmu = -(1/L^2) sum_k cos(k.r) exp(-xi tau)(1 - n_F)(tau - beta n_F)."""
    xi = dispersion(L, t, mu, alpha)
    tg = tau_grid(beta, n_tau)
    w = tau_weight(xi, tg, beta) * (tg[None, :] - beta * fermi(xi, beta)[:, None])
    return -(cos_kr(L) @ w) / (L * L)


def model_tables(model, deriv: bool = False) -> np.ndarray:
    """Tables for every flavor of `model` (inputs.Model), shape [nf][L^2][n_tau]."""
    f = dtable_dmu if deriv else table
    return np.stack([f(model.L, model.t, model.beta, model.mu[l], model.alpha[l], model.n_tau)
                     for l in range(model.n_flavors)])


def interp(tab: np.ndarray, r: int, dt: float, beta: float) -> float:
    """G(r, dt) for -beta < dt < beta from a table [L^2][n_tau]: linear
    interpolation on the grid; dt <= 0 maps to -G(r, dt + beta)."""
    n_tau = tab.shape[1]
    if dt > 0:
        s, tt = 1.0, dt
    else:
        s, tt = -1.0, dt + beta
    x = tt / beta * (n_tau - 1)
    m = min(int(np.floor(x)), n_tau - 2)
    f = x - m
    return s * ((1.0 - f) * tab[r, m] + f * tab[r, m + 1])


def displacement(si: int, sj: int, L: int) -> int:
    """Site index of r_i - r_j on the L x L torus (site = x + L y)."""
    dx = (si % L - sj % L) % L
    dy = (si // L - sj // L) % L
    return dx + L * dy


def gather_one(tabs: np.ndarray, sites, taus, L: int, beta: float) -> np.ndarray:
    """M[l][i][j] = G0_l(r_i - r_j, tau_i - tau_j) for one configuration."""
    n = len(sites)
    nf = tabs.shape[0]
    M = np.empty((nf, n, n))
    for l in range(nf):
        for i in range(n):
            for j in range(n):
                M[l, i, j] = interp(tabs[l], displacement(int(sites[i]), int(sites[j]), L),
                                    float(taus[i]) - float(taus[j]), beta)
    return M


def gather(tabs: np.ndarray, cfgs, L: int, beta: float, idx=None):
    """List of per-configuration matrices for inputs.Configs `cfgs`."""
    idx = range(cfgs.n_cfg) if idx is None else idx
    out = []
    for c in idx:
        o, n = int(cfgs.offset[c]), int(cfgs.order[c])
        out.append(gather_one(tabs, cfgs.site[o:o + n], cfgs.tau[o:o + n], L, beta))
    return out
