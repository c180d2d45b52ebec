"""torch.autograd Functions over the libcos forward and adjoint DP kernels.

* ``connected_sum(M, sigma, order, moff, ...)``: connected sums of explicit
  matrices; backward = the reverse (adjoint) DP kernel, giving dLoss/dM and
  dLoss/dsigma.
* ``connected_sum_model(mu, alpha, model, configs)``: connected sums from
  vertex coordinates; backward = adjoint DP + chain rule through the
  propagator tables, giving dLoss/dmu_l and dLoss/dalpha_l.
* ``connected_det(M, alpha, ...)``: SU(2) determinant-weight sums (the DP without
  cycle factors of Alg. 1); backward = its reverse sweep, dLoss/dM and dLoss/dalpha.
* ``connected_sum_bipartite(M4, sigma2, ...)`` and ``connected_det_bipartite(M4,
  alpha2, ...)``: the bipartite sums; backward = the bipartite reverse sweep.

PyTorch only holds tensors and streams here; every arithmetic step runs in the
CUDA kernels (no host fallback).
"""
from __future__ import annotations

import torch

from . import binding as B


class _ConnectedSum(torch.autograd.Function):
    @staticmethod
    def forward(ctx, M, sigma, order, moff, n_max, n_mat, loop_weight):
        sig = None if sigma is None else [float(s) for s in sigma.detach().cpu()]
        out = torch.empty(order.numel(), dtype=torch.float64, device=M.device)
        B.cos_connected_sum_matrices(n_max, order, moff, n_mat, loop_weight, sig, M.detach().contiguous(), "fp64",
                                     out)
        ctx.save_for_backward(M, order, moff)
        ctx.sig = sig
        ctx.sigma_shape = None if sigma is None else sigma.shape
        ctx.args = (n_max, n_mat, loop_weight)
        return out

    @staticmethod
    def backward(ctx, gout):
        M, order, moff = ctx.saved_tensors
        n_max, n_mat, loop_weight = ctx.args
        gM = torch.zeros_like(M)
        need_sig = ctx.sigma_shape is not None and ctx.needs_input_grad[1]
        gsig = torch.zeros(order.numel(), n_mat, dtype=torch.float64, device=M.device) if need_sig else None
        B.cos_connected_sum_matrices_grad(n_max, order, moff, n_mat, loop_weight, ctx.sig, M.detach().contiguous(),
                                          gout.detach().to(torch.float64).contiguous(), None, gM, gsig)
        gs = gsig.sum(0).to("cpu").reshape(ctx.sigma_shape) if need_sig else None
        return gM, gs, None, None, None, None, None


def connected_sum(M, sigma, order, moff, n_max: int, n_mat: int, loop_weight: int = 1):
    """Connected sums c[cfg] of packed matrices M (flat, blocks [n_mat][n][n] at moff[cfg]).
    sigma: CPU tensor of n_mat shift weights (may require grad) or None."""
    return _ConnectedSum.apply(M, sigma, order, moff, n_max, n_mat, loop_weight)


class _ConnectedSumModel(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, alpha, model, d_cfgs, n_max):
        tabs = B.cos_build_propagators(model.L, model.t, model.beta, model.U, [float(x) for x in mu],
                                       [float(x) for x in alpha], model.n_tau)
        order, offset, site, tau = d_cfgs
        out = torch.empty(order.numel(), dtype=torch.float64, device=order.device)
        B.cos_connected_sum_batch(tabs, n_max, order, offset, site, tau, "fp64", out)
        ctx.tabs = tabs
        ctx.d_cfgs = d_cfgs
        ctx.n_max = n_max
        ctx.nf = len(mu)
        return out

    @staticmethod
    def backward(ctx, gout):
        order, offset, site, tau = ctx.d_cfgs
        n = order.numel()
        gmu = torch.empty(n, ctx.nf, dtype=torch.float64, device=order.device)
        gal = torch.empty_like(gmu)
        B.cos_connected_sum_grad(ctx.tabs, ctx.n_max, order, offset, site, tau,
                                 gout.detach().to(torch.float64).contiguous(), gmu=gmu, galpha=gal)
        ctx.tabs.close()
        return gmu.sum(0).cpu(), gal.sum(0).cpu(), None, None, None


def connected_sum_model(mu, alpha, model, d_cfgs, n_max: int):
    """Connected sums from vertex coordinates for chemical potentials mu and shifts alpha
    (CPU tensors of n_flavors values, differentiable); other model fields from `model`."""
    return _ConnectedSumModel.apply(mu, alpha, model, d_cfgs, n_max)


def _host_list(t):
    return None if t is None else [float(x) for x in t.detach().cpu().reshape(-1)]


def _host_rows(t):
    return None if t is None else [[float(x) for x in row] for row in t.detach().cpu().reshape(-1, 2)]


class _ConnectedDet(torch.autograd.Function):
    @staticmethod
    def forward(ctx, M, alpha, order, moff, n_max):
        al = _host_list(alpha)
        out = torch.empty(order.numel(), dtype=torch.float64, device=M.device)
        B.cos_connected_det_matrices(n_max, order, moff, al, M.detach().contiguous(), "fp64", out)
        ctx.save_for_backward(M, order, moff)
        ctx.al = al
        ctx.alpha_shape = None if alpha is None else alpha.shape
        ctx.n_max = n_max
        return out

    @staticmethod
    def backward(ctx, gout):
        M, order, moff = ctx.saved_tensors
        gM = torch.zeros_like(M)
        need_al = ctx.alpha_shape is not None and ctx.needs_input_grad[1]
        gal = torch.zeros(order.numel(), 2, dtype=torch.float64, device=M.device) if need_al else None
        B.cos_connected_det_matrices_grad(ctx.n_max, order, moff, ctx.al, M.detach().contiguous(),
                                          gout.detach().to(torch.float64).contiguous(), None, gM, gal)
        ga = gal.sum(0).to("cpu").reshape(ctx.alpha_shape) if need_al else None
        return gM, ga, None, None, None


def connected_det(M, alpha, order, moff, n_max: int):
    """SU(2) determinant-weight connected sums of packed spin blocks M (flat, [2][n][n] at
    moff[cfg]); alpha: CPU tensor of the two diagonal shifts (may require grad) or None."""
    return _ConnectedDet.apply(M, alpha, order, moff, n_max)


class _ConnectedDetModel(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, alpha, model, d_cfgs, n_max):
        tabs = B.cos_build_propagators(model.L, model.t, model.beta, model.U, [float(x) for x in mu], [0.0, 0.0],
                                       model.n_tau)
        order, offset, site, tau = d_cfgs
        al = _host_list(alpha)
        out = torch.empty(order.numel(), dtype=torch.float64, device=order.device)
        B.cos_connected_det_batch(tabs, n_max, order, offset, site, tau, al, "fp64", out)
        ctx.tabs = tabs
        ctx.al = al
        ctx.d_cfgs = d_cfgs
        ctx.n_max = n_max
        return out

    @staticmethod
    def backward(ctx, gout):
        order, offset, site, tau = ctx.d_cfgs
        n = order.numel()
        gmu = torch.empty(n, 2, dtype=torch.float64, device=order.device)
        gal = torch.empty_like(gmu)
        B.cos_connected_det_grad(ctx.tabs, ctx.n_max, order, offset, site, tau, ctx.al,
                                 gout.detach().to(torch.float64).contiguous(), gmu=gmu, galpha=gal)
        ctx.tabs.close()
        return gmu.sum(0).cpu(), gal.sum(0).cpu(), None, None, None


def connected_det_model(mu, alpha, model, d_cfgs, n_max: int):
    """SU(2) determinant-weight connected sums from vertex coordinates for the spin chemical
    potentials mu and the diagonal shifts alpha (CPU tensors of 2 values, differentiable); the
    tables are built at mu with no dispersion shift; other model fields from `model`."""
    return _ConnectedDetModel.apply(mu, alpha, model, d_cfgs, n_max)


class _ConnectedBipartite(torch.autograd.Function):
    @staticmethod
    def forward(ctx, M4, sig2, order, moff, n_max, n_mat, loop_weight, det):
        s2 = _host_rows(sig2)
        out = torch.empty(order.numel(), dtype=torch.float64, device=M4.device)
        if det:
            B.cos_connected_det_bipartite_matrices(n_max, order, moff, s2, M4.detach().contiguous(), "fp64", out)
        else:
            B.cos_connected_sum_bipartite_matrices(n_max, order, moff, n_mat, loop_weight, s2,
                                                   M4.detach().contiguous(), "fp64", out)
        ctx.save_for_backward(M4, order, moff)
        ctx.s2 = s2
        ctx.sig_shape = None if sig2 is None else sig2.shape
        ctx.args = (n_max, n_mat, loop_weight, det)
        return out

    @staticmethod
    def backward(ctx, gout):
        M4, order, moff = ctx.saved_tensors
        n_max, n_mat, loop_weight, det = ctx.args
        gM = torch.zeros_like(M4)
        need_s = ctx.sig_shape is not None and ctx.needs_input_grad[1]
        gs = torch.zeros(order.numel(), n_mat, 2, dtype=torch.float64, device=M4.device) if need_s else None
        g = gout.detach().to(torch.float64).contiguous()
        if det:
            B.cos_connected_det_bipartite_matrices_grad(n_max, order, moff, ctx.s2, M4.detach().contiguous(), g,
                                                        None, gM, gs)
        else:
            B.cos_connected_sum_bipartite_matrices_grad(n_max, order, moff, n_mat, loop_weight, ctx.s2,
                                                        M4.detach().contiguous(), g, None, gM, gs)
        gsig = gs.sum(0).to("cpu").reshape(ctx.sig_shape) if need_s else None
        return gM, gsig, None, None, None, None, None, None


def connected_sum_bipartite(M4, sigma2, order, moff, n_max: int, n_mat: int, loop_weight: int = 1):
    """Bipartite connected sums of packed M4 blocks ([n_mat][2n][2n] at moff[cfg]); sigma2: CPU
    tensor [n_mat][2] of shift weights (may require grad) or None.  Orders up to 9, as the forward."""
    return _ConnectedBipartite.apply(M4, sigma2, order, moff, n_max, n_mat, loop_weight, False)


def connected_det_bipartite(M4, alpha2, order, moff, n_max: int):
    """Bipartite SU(2) determinant-weight sums of packed M4 blocks ([2][2n][2n] at moff[cfg]);
    alpha2: CPU tensor [2][2] of diagonal shifts (may require grad) or None."""
    return _ConnectedBipartite.apply(M4, alpha2, order, moff, n_max, 2, 1, True)


class _ConnectedBipartiteModel(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, alpha, model, d_cfgs, n_max):
        tabs = B.cos_build_propagators_honeycomb(model.L, model.t, model.beta, model.U, [float(x) for x in mu],
                                                 [float(x) for x in alpha], list(model.delta), model.n_tau)
        order, offset, site, tau = d_cfgs
        out = torch.empty(order.numel(), dtype=torch.float64, device=order.device)
        B.cos_connected_sum_bipartite_batch(tabs, n_max, order, offset, site, tau, "fp64", out)
        ctx.tabs = tabs
        ctx.d_cfgs = d_cfgs
        ctx.n_max = n_max
        ctx.nf = len(mu)
        return out

    @staticmethod
    def backward(ctx, gout):
        order, offset, site, tau = ctx.d_cfgs
        gmu = torch.empty(order.numel(), ctx.nf, dtype=torch.float64, device=order.device)
        gal = torch.empty_like(gmu)
        B.cos_connected_sum_bipartite_grad(ctx.tabs, ctx.n_max, order, offset, site, tau,
                                           gout.detach().to(torch.float64).contiguous(), gmu=gmu, galpha=gal)
        ctx.tabs.close()
        return gmu.sum(0).cpu(), gal.sum(0).cpu(), None, None, None


def connected_sum_bipartite_model(mu, alpha, model, d_cfgs, n_max: int):
    """Bipartite (honeycomb) connected sums from vertex coordinates for chemical potentials mu
    and uniform shifts alpha (CPU tensors of n_flavors values, differentiable); the staggered
    shifts delta and the other fields from the inputs.HoneycombModel `model`."""
    return _ConnectedBipartiteModel.apply(mu, alpha, model, d_cfgs, n_max)


class _ConnectedDetBipartiteModel(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, alpha2, model, d_cfgs, n_max):
        tabs = B.cos_build_propagators_honeycomb(model.L, model.t, model.beta, model.U, [float(x) for x in mu],
                                                 [0.0, 0.0], list(model.delta), model.n_tau)
        order, offset, site, tau = d_cfgs
        al = _host_rows(alpha2)
        out = torch.empty(order.numel(), dtype=torch.float64, device=order.device)
        B.cos_connected_det_bipartite_batch(tabs, n_max, order, offset, site, tau, al, "fp64", out)
        ctx.tabs = tabs
        ctx.al = al
        ctx.d_cfgs = d_cfgs
        ctx.n_max = n_max
        return out

    @staticmethod
    def backward(ctx, gout):
        order, offset, site, tau = ctx.d_cfgs
        n = order.numel()
        gmu = torch.empty(n, 2, dtype=torch.float64, device=order.device)
        gal = torch.empty(n, 2, 2, dtype=torch.float64, device=order.device)
        B.cos_connected_det_bipartite_grad(ctx.tabs, ctx.n_max, order, offset, site, tau, ctx.al,
                                           gout.detach().to(torch.float64).contiguous(), gmu=gmu, galpha2=gal)
        ctx.tabs.close()
        return gmu.sum(0).cpu(), gal.sum(0).cpu(), None, None, None


def connected_det_bipartite_model(mu, alpha2, model, d_cfgs, n_max: int):
    """Bipartite determinant-weight connected sums from vertex coordinates for the spin chemical
    potentials mu (CPU tensor of 2 values) and the diagonal shifts alpha2 (CPU tensor [2][2],
    spin then sublattice), both differentiable; the honeycomb tables are built at mu with the
    staggered shifts delta of the inputs.HoneycombModel `model` and no uniform shift."""
    return _ConnectedDetBipartiteModel.apply(mu, alpha2, model, d_cfgs, n_max)
