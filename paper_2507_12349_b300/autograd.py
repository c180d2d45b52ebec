"""torch.autograd Functions over the libcos forward and adjoint DP kernels.

* ``connected_sum(M, sigma, order, moff, ...)``: connected sums of explicit
  matrices; backward = the reverse (adjoint) DP kernel, giving dLoss/dM and
  dLoss/dsigma.
* ``connected_sum_model(mu, alpha, model, configs)``: connected sums from
  vertex coordinates; backward = adjoint DP + chain rule through the
  propagator tables, giving dLoss/dmu_l and dLoss/dalpha_l.

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
