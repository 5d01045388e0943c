"""FP64 CPU oracle for the borehole FWI hot path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path (the
CUDA library and its binding) never imports this module.

The wave-equation parts (forward modelling of Eq. 2, the adjoint of Eq. 6 as
the literal transpose of the discrete forward, and the correlations of Eq. 7
and Eq. 8) live in ``bh_oracle.c``; this module loads it with ctypes and adds
the plain elementwise steps in numpy:

- data residual and misfit, Eq. 5 and Eq. 1;
- the diagonal preconditioner (Numerical Examples, Fig. 6; the paper gives no
  formula, the reading used is a Shin-style pseudo-Hessian, see
  ``precondition``);
- the gradient-descent update of Eq. 9 and Eq. 10 with the step chosen to
  bound the largest relative model change, then Eq. 11 and Eq. 12;
- the chain rule to (Vp, Vs) and the multi-shot sum.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bh_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")

NFIELD = 6
NACC = 8
ACC_NAMES = ("G_lam", "G_munn", "G_murz", "G_br", "G_bz", "H_lam", "H_munn", "H_murz")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP on the forward loops)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [
        ("nr", ctypes.c_int), ("nz", ctypes.c_int), ("nt", ctypes.c_int),
        ("npml_r", ctypes.c_int), ("npml_z", ctypes.c_int),
        ("dr", ctypes.c_double), ("dz", ctypes.c_double), ("dt", ctypes.c_double),
        ("f0", ctypes.c_double), ("pml_R", ctypes.c_double), ("vpmax", ctypes.c_double),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        gp = ctypes.POINTER(_Grid)
        _lib.orc_forward.argtypes = [gp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ip, dp, dp, dp]
        _lib.orc_forward.restype = ctypes.c_int
        _lib.orc_adjoint.argtypes = [gp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ip, dp, dp, dp, dp]
        _lib.orc_adjoint.restype = ctypes.c_int
        _lib.orc_finalize.argtypes = [gp, dp, dp, dp, dp, dp]
        _lib.orc_finalize.restype = ctypes.c_int
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


@dataclass
class Grid:
    """One simulation window: nr x nz cells (C-PML included), nt steps."""
    nr: int
    nz: int
    nt: int
    npml_r: int
    npml_z: int
    dr: float
    dz: float
    dt: float
    f0: float
    pml_R: float = 1e-3

    def c(self, vpmax: float) -> _Grid:
        return _Grid(self.nr, self.nz, self.nt, self.npml_r, self.npml_z, self.dr, self.dz,
                     self.dt, self.f0, self.pml_R, float(vpmax))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def forward(grid: Grid, vp, vs, rho, wavelet, src, rec_iz, *, vpmax=None, store_v=True,
            force=None):
    """Forward modelling of Eq. 2 on one window.

    Returns (seis [nrec, nt], vhist [nt, 2, nr*nz] or None)."""
    lib = _load()
    vp, vs, rho, wavelet = _f64(vp), _f64(vs), _f64(rho), _f64(wavelet)
    rec = np.ascontiguousarray(rec_iz, dtype=np.int32)
    vpmax = float(vp.max()) if vpmax is None else float(vpmax)
    nc = grid.nr * grid.nz
    seis = np.zeros((len(rec), grid.nt))
    vhist = np.zeros((grid.nt, 2, nc)) if store_v else None
    if force is not None:
        force = _f64(force)
        assert force.shape == (grid.nt, NFIELD, nc)
    g = grid.c(vpmax)
    rc = lib.orc_forward(ctypes.byref(g), _dp(vp), _dp(vs), _dp(rho), _dp(wavelet),
                         int(src[0]), int(src[1]), len(rec), _ip(rec), _dp(seis), _dp(vhist),
                         _dp(force))
    if rc != 0:
        raise MemoryError("oracle forward: allocation failed")
    return seis, vhist


def adjoint(grid: Grid, vp, vs, rho, resid, src, rec_iz, vhist, *, vpmax=None,
            want_wavelet_bar=False, want_force_bar=False):
    """Adjoint modelling (discrete Eq. 6) and correlation accumulators.

    Returns (acc [NACC, nr*nz], wavelet_bar [nt] or None, force_bar or None)."""
    lib = _load()
    vp, vs, rho, resid = _f64(vp), _f64(vs), _f64(rho), _f64(resid)
    rec = np.ascontiguousarray(rec_iz, dtype=np.int32)
    vpmax = float(vp.max()) if vpmax is None else float(vpmax)
    nc = grid.nr * grid.nz
    acc = np.zeros((NACC, nc))
    wbar = np.zeros(grid.nt) if want_wavelet_bar else None
    fbar = np.zeros((grid.nt, NFIELD, nc)) if want_force_bar else None
    g = grid.c(vpmax)
    rc = lib.orc_adjoint(ctypes.byref(g), _dp(vp), _dp(vs), _dp(rho), _dp(resid),
                         int(src[0]), int(src[1]), len(rec), _ip(rec), _dp(_f64(vhist)),
                         _dp(acc), _dp(wbar), _dp(fbar))
    if rc != 0:
        raise MemoryError("oracle adjoint: allocation failed")
    return acc, wbar, fbar


def finalize(grid: Grid, vp, vs, rho, acc, *, vpmax=None):
    """Per-cell gradients and pseudo-Hessians from the accumulators.

    Returns dict with g_lam, g_mu, g_rho, H_lam, H_mu, each [nr, nz]."""
    lib = _load()
    vp, vs, rho = _f64(vp), _f64(vs), _f64(rho)
    vpmax = float(vp.max()) if vpmax is None else float(vpmax)
    nc = grid.nr * grid.nz
    out = np.zeros((5, nc))
    g = grid.c(vpmax)
    rc = lib.orc_finalize(ctypes.byref(g), _dp(vp), _dp(vs), _dp(rho), _dp(_f64(acc)),
                          _dp(out))
    if rc != 0:
        raise MemoryError("oracle finalize: allocation failed")
    names = ("g_lam", "g_mu", "g_rho", "H_lam", "H_mu")
    return {k: out[q].reshape(grid.nr, grid.nz) for q, k in enumerate(names)}


# ---------------------------------------------------------------------------
# Elementwise steps (numpy, FP64)


def lame(vp, vs, rho):
    """Eq. 3 and Eq. 4: lambda = rho Vp^2 - 2 rho Vs^2, mu = rho Vs^2."""
    vp, vs, rho = _f64(vp), _f64(vs), _f64(rho)
    return rho * vp * vp - 2.0 * rho * vs * vs, rho * vs * vs


def velocities(lam, mu, rho):
    """Eq. 11 and Eq. 12."""
    return np.sqrt((lam + 2.0 * mu) / rho), np.sqrt(mu / rho)


def residual_misfit(seis_mod, seis_obs):
    """Eq. 5 (residual) and Eq. 1 (J = 1/2 ||p_mod - p_mes||^2, no dt weight)."""
    resid = _f64(seis_mod) - _f64(seis_obs)
    return resid, 0.5 * float(np.sum(resid * resid))


def precondition(g, H, mask, eps_rel):
    """Diagonal preconditioner (reading): g / (H + eps * max_mask H), zero
    outside the inversion mask (fluid and C-PML cells)."""
    g, H = _f64(g), _f64(H)
    hmax = float(H[mask].max()) if mask.any() else 0.0
    out = np.zeros_like(g)
    denom = H + eps_rel * hmax
    ok = mask & (denom > 0)
    out[ok] = g[ok] / denom[ok]
    return out


def update(lam, mu, rho, g_lam, g_mu, mask, kappa):
    """Eq. 9 and Eq. 10 with alpha_m = kappa max|m| / max|g_m| over the mask,
    so that no cell changes by more than kappa of the largest modulus; then
    mu >= 0, Vp >= 1 m/s, and Eq. 11 / Eq. 12.

    Returns (lam_new, mu_new, vp_new, vs_new, (alpha_lam, alpha_mu))."""
    lam, mu, rho = _f64(lam).copy(), _f64(mu).copy(), _f64(rho)
    alphas = []
    for m, gm in ((lam, g_lam), (mu, g_mu)):
        gmax = float(np.abs(gm[mask]).max()) if mask.any() else 0.0
        mmax = float(np.abs(m[mask]).max()) if mask.any() else 0.0
        alphas.append(kappa * mmax / gmax if gmax > 0 else 0.0)
    lam[mask] -= alphas[0] * _f64(g_lam)[mask]
    mu[mask] -= alphas[1] * _f64(g_mu)[mask]
    mu = np.maximum(mu, 0.0)
    floor = rho * 1.0 - 2.0 * mu  # lambda + 2 mu >= rho (1 m/s)^2
    lam = np.where(lam < floor, floor, lam)
    vp, vs = velocities(lam, mu, rho)
    return lam, mu, vp, vs, tuple(alphas)


def chain_to_velocity(g_lam, g_mu, g_rho, vp, vs, rho):
    """Gradients with respect to (Vp, Vs, rho) from those with respect to
    (lambda, mu, rho), by Eq. 3 and Eq. 4."""
    vp, vs, rho = _f64(vp), _f64(vs), _f64(rho)
    g_vp = 2.0 * rho * vp * g_lam
    g_vs = 2.0 * rho * vs * (g_mu - 2.0 * g_lam)
    g_rho_v = g_rho + (vp * vp - 2.0 * vs * vs) * g_lam + vs * vs * g_mu
    return g_vp, g_vs, g_rho_v


def update_velocity(vp, vs, rho, g_lam, g_mu, g_rho, mask, kappa, update_rho=False):
    """Eq. 9 and Eq. 10 taken in the velocities (and, with update_rho, the
    density) instead of the Lame parameters: the gradients with respect to
    (Vp, Vs, rho) come from those with respect to (lambda, mu, rho) by the
    chain rule of Eq. 3 and Eq. 4 (chain_to_velocity; g_rho None means rho
    has no gradient of its own), each parameter steps by
    alpha_m = kappa max|m| / max|g_m| over the mask, then Vs >= 0,
    Vp >= 1 m/s, rho >= 1 kg/m^3, and lambda, mu follow from Eq. 3, Eq. 4.

    Returns (vp, vs, rho, lam, mu, (alpha_vp, alpha_vs, alpha_rho))."""
    vp, vs, rho = _f64(vp).copy(), _f64(vs).copy(), _f64(rho).copy()
    g_rho = np.zeros_like(vp) if g_rho is None else _f64(g_rho)
    g_vp, g_vs, g_rho_v = chain_to_velocity(g_lam, g_mu, g_rho, vp, vs, rho)
    steps = [(vp, g_vp), (vs, g_vs)] + ([(rho, g_rho_v)] if update_rho else [])
    alphas = [0.0, 0.0, 0.0]
    for q, (m, gm) in enumerate(steps):
        gmax = float(np.abs(gm[mask]).max()) if mask.any() else 0.0
        mmax = float(np.abs(m[mask]).max()) if mask.any() else 0.0
        alphas[q] = kappa * mmax / gmax if gmax > 0 else 0.0
    for q, (m, gm) in enumerate(steps):
        m[mask] -= alphas[q] * gm[mask]
    vs = np.maximum(vs, 0.0)
    vp = np.maximum(vp, 1.0)
    rho = np.maximum(rho, 1.0)
    lam, mu = lame(vp, vs, rho)
    return vp, vs, rho, lam, mu, tuple(alphas)


def starting_model(nr, dr, r_wall, r_far, vp_wall, vs_wall, vp_far, vs_far, vp_fluid):
    """Starting model of the Numerical Examples (Fig. 3, Fig. 4): per depth,
    the P and S velocities at the borehole wall (from the near-monopole data)
    and at r_far (one meter into the formation, from the ultra-far-monopole
    data), linear in r in between, the far values beyond r_far, and the
    borehole fluid (Vs = 0) in the cells whose centre lies inside r_wall.
    vp_wall, vs_wall, vp_far, vs_far: [nz].  Returns (vp, vs) [nr, nz]."""
    r = (np.arange(nr) + 0.5) * dr
    t = np.clip((r - r_wall) / (r_far - r_wall), 0.0, 1.0)[:, None]
    vpw, vsw, vpf, vsf = (_f64(a)[None, :] for a in (vp_wall, vs_wall, vp_far, vs_far))
    vp = vpw + t * (vpf - vpw)
    vs = vsw + t * (vsf - vsw)
    fluid = r < r_wall
    vp[fluid, :] = vp_fluid
    vs[fluid, :] = 0.0
    return vp, vs


def inversion_mask(nr, nz, npml_r, npml_z, vs, windows=None):
    """Cells that are unknowns: formation cells (Vs > 0) outside the radial
    C-PML and inside the axial interior (outside the top and bottom C-PML) of
    at least one shot window.  windows: list of (z_offset, nz_window); None
    means one window covering the whole model."""
    if windows is None:
        windows = [(0, nz)]
    cols = np.zeros(nz, dtype=bool)
    for z0, nzs in windows:
        cols[z0 + npml_z: z0 + nzs - npml_z] = True
    m = np.zeros((nr, nz), dtype=bool)
    m[: nr - npml_r, :] = cols[None, :]
    return m & (np.asarray(vs).reshape(nr, nz) > 0)


# ---------------------------------------------------------------------------
# Multi-shot driver: every shot simulates its own axial window of the global
# model and adds its gradient to the global one.


def shot_gradient(grid: Grid, vp, vs, rho, wavelet, shots, seis_obs):
    """Forward, residual, adjoint and gradient over all shots.

    vp, vs, rho: [nr, nz_global]; shots: list of dicts with z_offset, nz,
    src (ir, iz) and rec_iz (window coordinates); seis_obs: [nshots, nrec, nt].
    Returns dict with J, resid [nshots], seis [nshots], and global g_lam,
    g_mu, g_rho, H_lam, H_mu [nr, nz_global]."""
    vp, vs, rho = _f64(vp), _f64(vs), _f64(rho)
    nr, nzg = vp.shape
    vpmax = float(vp.max())
    out = {k: np.zeros((nr, nzg)) for k in ("g_lam", "g_mu", "g_rho", "H_lam", "H_mu")}
    J = 0.0
    seis_all, resid_all = [], []
    for s, sh in enumerate(shots):
        z0, nzs = sh["z_offset"], sh["nz"]
        sl = np.s_[:, z0: z0 + nzs]
        g = Grid(nr, nzs, grid.nt, grid.npml_r, grid.npml_z, grid.dr, grid.dz, grid.dt,
                 grid.f0, grid.pml_R)
        w = [np.ascontiguousarray(a[sl]) for a in (vp, vs, rho)]
        seis, vh = forward(g, *w, wavelet, sh["src"], sh["rec_iz"], vpmax=vpmax)
        resid, Js = residual_misfit(seis, seis_obs[s])
        acc, _, _ = adjoint(g, *w, resid, sh["src"], sh["rec_iz"], vh, vpmax=vpmax)
        del vh
        fin = finalize(g, *w, acc, vpmax=vpmax)
        for k in out:
            out[k][sl] += fin[k]
        J += Js
        seis_all.append(seis)
        resid_all.append(resid)
    out["J"] = J
    out["seis"] = seis_all
    out["resid"] = resid_all
    return out
