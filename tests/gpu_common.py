"""Shared helpers of the GPU tests: run the CUDA path through the C ABI and
the oracle on the same seeded inputs, and compare."""
import numpy as np
import torch

from oracle import oracle as O


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a))


def oracle_grid(w):
    return O.Grid(w.nr, w.nz, w.nt, w.npml_r, w.npml_z, w.dr, w.dz, w.dt, w.f0, w.pml_R)


def oracle_observed(w):
    """'Measured' data: oracle forward modelling in the true model."""
    obs = []
    vpmax = float(w.vp.max())
    for sh in w.shots:
        z0, nzs = sh["z_offset"], sh["nz"]
        sl = np.s_[:, z0: z0 + nzs]
        g = O.Grid(w.nr, nzs, w.nt, w.npml_r, w.npml_z, w.dr, w.dz, w.dt, w.f0, w.pml_R)
        s, _ = O.forward(g, *(np.ascontiguousarray(a[sl]) for a in (w.vp_true, w.vs_true,
                                                                      w.rho_true)),
                         w.wavelet, sh["src"], sh["rec_iz"], store_v=False, vpmax=vpmax)
        obs.append(s)
    nrec = max(len(sh["rec_iz"]) for sh in w.shots)
    out = np.zeros((len(w.shots), nrec, w.nt))
    for k, s in enumerate(obs):
        out[k, : s.shape[0]] = s
    return out


def gpu_gradient(w, obs, device="cuda", options=None):
    """Forward, residual, adjoint through libbh (bh_set_option for every item
    of `options` first).  Returns the model and a dict of numpy arrays."""
    from paper_2005_00281_gb300.bh import model_from_workload

    m = model_from_workload(w, device=device)
    for k, v in (options or {}).items():
        m.set_option(k, v)
    wav = torch.from_numpy(w.wavelet).to(device)
    seis = m.forward(wav)
    obs_t = torch.from_numpy(obs.astype(np.float32)).to(device)
    resid, J = m.residual_misfit(seis, obs_t)
    g_lam, g_mu, g_rho = m.adjoint_gradient(resid)
    H_lam, H_mu = m.hessian()
    torch.cuda.synchronize()
    out = dict(seis=seis.cpu().numpy(), resid=resid.cpu().numpy(), J=J, g_lam=g_lam.cpu().numpy(),
               g_mu=g_mu.cpu().numpy(), g_rho=g_rho.cpu().numpy(), H_lam=H_lam.cpu().numpy(),
               H_mu=H_mu.cpu().numpy())
    return m, out


def oracle_gradient(w, obs):
    """The oracle on the same inputs (obs is what the GPU path was given,
    rounded to float32 like the GPU copy)."""
    obs32 = obs.astype(np.float32).astype(np.float64)
    return O.shot_gradient(oracle_grid(w), w.vp, w.vs, w.rho, w.wavelet, w.shots, obs32)


def regions(w):
    """Named index sets of one window (window = global model): the axis row,
    the rows on both sides of the fluid-solid wall, the last rows and columns
    before the C-PML, and the neighbourhoods of the source and of every
    receiver.  Relative errors over a whole array can hide a wrong band of
    small values; these are checked one by one."""
    nr, nz, pr, pz = w.nr, w.nz, w.npml_r, w.npml_z
    fl = int(np.argmax(w.vs[:, nz // 2] > 0))      # first formation row
    sh = w.shots[0]
    si, sj = sh["src"]
    out = {
        "axis": np.s_[0:1, pz: nz - pz],
        "wall": np.s_[max(fl - 1, 0): fl + 1, pz: nz - pz],
        "radial_pml_edge": np.s_[nr - pr - 2: nr - pr, pz: nz - pz],
        "top_pml_edge": np.s_[0: nr - pr, pz: pz + 2],
        "bottom_pml_edge": np.s_[0: nr - pr, nz - pz - 2: nz - pz],
        "source": np.s_[max(si - 3, 0): si + 4, max(sj - 3, pz): min(sj + 4, nz - pz)],
    }
    for k, rj in enumerate(sh["rec_iz"]):
        out[f"receiver{k}"] = np.s_[0:3, max(rj - 2, pz): min(rj + 3, nz - pz)]
    return out


def region_errors(w, a, b):
    """{region: relative L2 error of a against b over the region} for the
    regions where b is not zero."""
    out = {}
    for name, sl in regions(w).items():
        ref = np.asarray(b)[sl]
        if np.linalg.norm(ref) > 0:
            out[name] = rel_l2(np.asarray(a)[sl], ref)
    return out


def max_abs_error(a, b):
    """max |a - b| / max |b|"""
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - b)) / np.max(np.abs(b)))
