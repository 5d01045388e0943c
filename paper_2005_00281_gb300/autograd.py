"""Differentiable forward modelling and misfit.

    seis = BhWave.apply(vp, vs, rho, model, wavelet)
    J = BhMisfit.apply(seis, seis_obs, model)

BhWave's backward is libbh's discrete adjoint (Eq. 6, the exact transpose of
the forward step) with the fused Eq. 7 / Eq. 8 correlations; `grad_output`
of the seismograms is the adjoint source.  It returns float32 gradients with
respect to Vp, Vs and rho (the chain rule runs in the library).  BhMisfit is
Eq. 1 and Eq. 5 through bh_residual_misfit: its value is the library's FP64
misfit and its gradient the library's residual.  Nothing of the method is
computed in PyTorch here.
"""
from __future__ import annotations

import torch


class BhWave(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vp, vs, rho, model, wavelet):
        model.set_model(vp.contiguous(), vs.contiguous(), rho.contiguous())
        seis = model.forward(wavelet.contiguous())
        ctx.model = model
        # the model keeps one forward history; backward must find this one
        ctx.version = model.info("state_version")
        return seis

    @staticmethod
    def backward(ctx, grad_seis):
        m = ctx.model
        if m.info("state_version") != ctx.version:
            raise RuntimeError("BhWave.backward: the model ran another forward, set_model or "
                               "update since this forward; its stored history is not this "
                               "graph's (run backward before reusing the model)")
        g_lam, g_mu, g_rho = m.adjoint_gradient(grad_seis.contiguous().float(), with_rho=True)
        g_vp, g_vs, g_rho_v = m.velocity_gradient(g_lam, g_mu, g_rho)
        return g_vp, g_vs, g_rho_v, None, None


class BhMisfit(torch.autograd.Function):
    """J = 1/2 ||seis - seis_obs||^2 (Eq. 1) in FP64 by the library; dJ/dseis
    is the residual of Eq. 5 the library returns with it."""

    @staticmethod
    def forward(ctx, seis, seis_obs, model):
        resid, J = model.residual_misfit(seis.detach().contiguous(),
                                         seis_obs.detach().contiguous())
        ctx.save_for_backward(resid)
        return torch.tensor(J, dtype=torch.float64, device=seis.device)

    @staticmethod
    def backward(ctx, grad_J):
        (resid,) = ctx.saved_tensors
        return (grad_J.to(resid.dtype) * resid), None, None


def misfit(seis, seis_obs, model):
    """Eq. 1, differentiable, computed by the library (bh_residual_misfit)."""
    return BhMisfit.apply(seis, seis_obs, model)
