"""Gradient-descent FWI driver (Method section, Fig. 1): forward modelling,
data residual, adjoint modelling with the gradient correlation, diagonal
preconditioning, model update, repeated until the misfit falls below a
threshold or an iteration cap.  Every step runs in libbh; this loop only
sequences the calls and keeps the history.  Resumable from an .npz."""
from __future__ import annotations

import os
import time
from dataclasses import dataclass, field

import numpy as np
import torch


@dataclass
class FwiState:
    iteration: int = 0
    J: list = field(default_factory=list)
    alpha: list = field(default_factory=list)
    seconds: list = field(default_factory=list)


def save(path, model, state: FwiState, rho):
    vp, vs = model.velocities()
    np.savez(path, vp=vp.cpu().numpy(), vs=vs.cpu().numpy(), rho=rho.cpu().numpy(),
             iteration=state.iteration, J=np.array(state.J), alpha=np.array(state.alpha),
             seconds=np.array(state.seconds))


def load(path, model, device="cuda"):
    d = np.load(path)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    rho = t(d["rho"])
    model.set_model(t(d["vp"]), t(d["vs"]), rho)
    st = FwiState(int(d["iteration"]), list(d["J"]), [tuple(a) for a in d["alpha"]],
                  list(d["seconds"]))
    return st, rho


def run(model, wavelet, seis_obs, iterations, *, kappa=0.02, eps_rel=1e-3, threshold=0.0,
        precondition=True, state: FwiState | None = None, checkpoint_path=None, rho=None,
        log=None):
    """Run up to `iterations` more inversion steps.  Returns the FwiState."""
    st = state or FwiState()
    seis = model.empty_seis()
    resid = torch.empty_like(seis)
    for _ in range(iterations):
        t0 = time.perf_counter()
        model.forward(wavelet, seis)
        _, J = model.residual_misfit(seis, seis_obs, resid)
        if J <= threshold:
            st.J.append(J)
            break
        g_lam, g_mu, _ = model.adjoint_gradient(resid, with_rho=False)
        if precondition:
            model.precondition(g_lam, g_mu, eps_rel)
        alpha, _, _ = model.update(g_lam, g_mu, kappa, want_velocities=False)
        st.iteration += 1
        st.J.append(J)
        st.alpha.append(alpha)
        st.seconds.append(time.perf_counter() - t0)
        if log:
            log(f"iteration {st.iteration}: J = {J:.6e}, alpha = {alpha[0]:.3e}, {alpha[1]:.3e}")
        if checkpoint_path and rho is not None:
            tmp = checkpoint_path + ".tmp.npz"
            save(tmp, model, st, rho)
            os.replace(tmp, checkpoint_path)
    return st
