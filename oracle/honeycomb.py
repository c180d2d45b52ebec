"""Two-band (honeycomb) free propagators and the bipartite gather.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Methods A, honeycomb lattice with nearest-neighbour hopping: per flavor l the Bloch
Hamiltonian on the two sublattices (A, B) of a unit cell is
    H_l(k) = [[ delta_l - (mu_l - alpha_l),  eps(k)                          ],
              [ conj(eps(k)),                -delta_l - (mu_l - alpha_l)     ]],
    eps(k) = -t (1 + exp(i k.b1) + exp(i k.b2)),
with k.b1 = 2 pi m_1 / L, k.b2 = 2 pi m_2 / L on an L x L torus of unit cells (cell
R = r_1 b1 + r_2 b2, site index r_1 + L r_2).  With G_{ss'}(R, tau) = -<T c_{R,s}(tau)
c^+_{0,s'}(0)> (the square lattice's sign convention),
    G_l(R, tau) = -(1/L^2) sum_k exp(i k.R) exp(-H_l(k) tau) (1 - n_F(H_l(k))),  0 < tau < beta,
a 2 x 2 matrix in the sublattice indices, real because the real-space hopping is real.
The matrix function is taken through numpy's Hermitian eigendecomposition (a library
primitive); the exponential weights use the same overflow-free forms as the square tables.

Readings shared with the square lattice: n_tau grid points tau_m = m beta / (n_tau - 1)
holding G(0^+) .. G(beta^-); linear interpolation; dt <= 0 reads -G(dt + beta).
"""
from __future__ import annotations

import numpy as np

from .propagators import displacement, tau_grid, tau_weight


def hc_momenta(L: int):
    """(k.b1, k.b2) for k index m_1 + L m_2."""
    m = np.arange(L)
    k1, k2 = np.meshgrid(2 * np.pi * m / L, 2 * np.pi * m / L, indexing="xy")
    return k1.ravel(), k2.ravel()


def hc_eps(L: int, t: float) -> np.ndarray:
    k1, k2 = hc_momenta(L)
    return -t * (1.0 + np.exp(1j * k1) + np.exp(1j * k2))


def hc_bloch(L: int, t: float, mu: float, alpha: float, delta: float) -> np.ndarray:
    """H(k) for every k, shape [L^2][2][2] (complex)."""
    eps = hc_eps(L, t)
    H = np.zeros((L * L, 2, 2), dtype=np.complex128)
    H[:, 0, 0] = delta - (mu - alpha)
    H[:, 1, 1] = -delta - (mu - alpha)
    H[:, 0, 1] = eps
    H[:, 1, 0] = np.conj(eps)
    return H


def hc_phase(L: int) -> np.ndarray:
    """exp(i k.R) for R = r_1 + L r_2 (rows) and k = m_1 + L m_2 (columns)."""
    k1, k2 = hc_momenta(L)
    r = np.arange(L * L)
    r1, r2 = r % L, r // L
    return np.exp(1j * (np.outer(r1, k1) + np.outer(r2, k2)))


def hc_table(L: int, t: float, beta: float, mu: float, alpha: float, delta: float, n_tau: int) -> np.ndarray:
    """G_{ss'}(R, tau_m) for 0^+ <= tau_m <= beta^-, shape [2][2][L^2][n_tau]."""
    H = hc_bloch(L, t, mu, alpha, delta)
    E, U = np.linalg.eigh(H)                                  # E [k][2], U [k][s][n]
    tg = tau_grid(beta, n_tau)
    w = np.stack([tau_weight(E[:, b], tg, beta) for b in range(2)], axis=1)   # [k][n][tau]
    P = hc_phase(L)
    out = np.empty((2, 2, L * L, n_tau))
    for s in range(2):
        for sp in range(2):
            F = np.einsum("kn,knm->km", U[:, s, :] * np.conj(U[:, sp, :]), w)   # [k][tau]
            out[s, sp] = -np.real(P @ F) / (L * L)
    return out


def hc_model_tables(model) -> np.ndarray:
    """Tables for every flavor of an inputs.HoneycombModel, shape [nf][2][2][L^2][n_tau]."""
    return np.stack([hc_table(model.L, model.t, model.beta, model.mu[l], model.alpha[l], model.delta[l],
                              model.n_tau) for l in range(model.n_flavors)])


def hc_interp(tab: np.ndarray, r: int, dt: float, beta: float) -> float:
    """Linear interpolation of one [L^2][n_tau] table at (r, dt), dt <= 0 -> -G(r, dt + beta)."""
    n_tau = tab.shape[1]
    if dt > 0:
        sg, tt = 1.0, dt
    else:
        sg, tt = -1.0, dt + beta
    x = tt / beta * (n_tau - 1)
    m = min(int(np.floor(x)), n_tau - 2)
    f = x - m
    return sg * ((1.0 - f) * tab[r, m] + f * tab[r, m + 1])


def hc_gather_one(tabs: np.ndarray, sites, taus, L: int, beta: float) -> np.ndarray:
    """M4[l][i][s][j][t] = G_l^{st}(R_i - R_j, tau_i - tau_j) for one configuration."""
    n = len(sites)
    nf = tabs.shape[0]
    M4 = np.empty((nf, n, 2, n, 2))
    for l in range(nf):
        for i in range(n):
            for j in range(n):
                r = displacement(int(sites[i]), int(sites[j]), L)
                dt = float(taus[i]) - float(taus[j])
                for s in range(2):
                    for t in range(2):
                        M4[l, i, s, j, t] = hc_interp(tabs[l, s, t], r, dt, beta)
    return M4


def hc_gather(tabs: np.ndarray, cfgs, L: int, beta: float, idx=None):
    idx = range(cfgs.n_cfg) if idx is None else idx
    out = []
    for c in idx:
        o, n = int(cfgs.offset[c]), int(cfgs.order[c])
        out.append(hc_gather_one(tabs, cfgs.site[o:o + n], cfgs.tau[o:o + n], L, beta))
    return out
