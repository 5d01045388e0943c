"""Differentiable forward modelling: a torch.autograd.Function whose backward
pass is libbh's discrete adjoint (Eq. 6, exact transpose of the forward
step) with the fused Eq. 7 / Eq. 8 correlations.

    seis = BhWave.apply(vp, vs, rho, model, wavelet)

`grad_output` of the seismograms is the adjoint source; for the misfit of
Eq. 1 it is the residual of Eq. 5.  The backward returns float32 gradients
with respect to Vp, Vs and rho (the chain rule runs in the library).
"""
from __future__ import annotations

import torch


class BhWave(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vp, vs, rho, model, wavelet):
        model.set_model(vp.contiguous(), vs.contiguous(), rho.contiguous())
        seis = model.forward(wavelet.contiguous())
        ctx.model = model
        return seis

    @staticmethod
    def backward(ctx, grad_seis):
        m = ctx.model
        g_lam, g_mu, g_rho = m.adjoint_gradient(grad_seis.contiguous().float(), with_rho=True)
        g_vp, g_vs, g_rho_v = m.velocity_gradient(g_lam, g_mu, g_rho)
        return g_vp, g_vs, g_rho_v, None, None


def misfit(seis, seis_obs):
    """Eq. 1, differentiable: J = 1/2 ||seis - seis_obs||^2 (FP64 sum)."""
    d = (seis - seis_obs).double()
    return 0.5 * torch.sum(d * d)
