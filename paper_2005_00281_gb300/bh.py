"""Thin ctypes binding of libbh (include/bh.h).

Argument marshalling only: every step of the path runs in the CUDA library.
Tensors are PyTorch CUDA tensors (device memory and streams); the library
enqueues on the stream that was current when the model was created.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import torch

from .build import LIB

BH_OK = 0
STATUS_NAMES = {0: "BH_OK", 1: "BH_ERR_INVALID_ARG", 2: "BH_ERR_CFL", 3: "BH_ERR_OOM",
                4: "BH_ERR_CUDA", 5: "BH_ERR_TIMEOUT", 6: "BH_ERR_STATE",
                7: "BH_ERR_UNSUPPORTED"}

# every entry point declared in include/bh.h
EXPORTS = ("bh_model_create", "bh_model_destroy", "bh_set_model", "bh_forward",
           "bh_residual_misfit", "bh_adjoint_gradient", "bh_get_hessian", "bh_precondition",
           "bh_update", "bh_get_model", "bh_status_string", "bh_last_error",
           "bh_profile_enable", "bh_profile_read", "bh_profile_reset",
           "bh_residual_misfit_noalloc", "bh_set_option", "bh_get_info",
           "bh_checkpoint_plan", "bh_velocity_gradient", "bh_update_velocity",
           "bh_get_density", "bh_plan_history", "bh_starting_model", "bh_tune",
           "bh_tune_lookup")
TUNE_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.txt")
NOALLOC_MAX_SAMPLES = 33554432
KERNELS = ("fwd_vel", "fwd_stress", "adj_stress", "adj_vel", "fwd_persist", "adj_persist",
           "fwd_step")


class BhError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("nr", ctypes.c_int), ("nz", ctypes.c_int), ("nt", ctypes.c_int),
        ("npml_r", ctypes.c_int), ("npml_z", ctypes.c_int),
        ("dr", ctypes.c_double), ("dz", ctypes.c_double), ("dt", ctypes.c_double),
        ("f0", ctypes.c_double), ("pml_R", ctypes.c_double),
        ("snapshot_precision", ctypes.c_int), ("checkpoint_cap_bytes", ctypes.c_size_t),
    ]


class ShotDesc(ctypes.Structure):
    _fields_ = [
        ("z_offset", ctypes.c_int), ("nz", ctypes.c_int),
        ("src_ir", ctypes.c_int), ("src_iz", ctypes.c_int),
        ("nrec", ctypes.c_int), ("rec_iz", ctypes.POINTER(ctypes.c_int)),
    ]


_lib = None


def load_library(path: str | None = None):
    """Load libbh.so; raises if it is missing (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libbh.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    st = ctypes.c_int
    lib.bh_model_create.argtypes = [ctypes.POINTER(GridDesc), ctypes.c_int, vp, vp, vp,
                                    ctypes.POINTER(ShotDesc), ctypes.c_int, vp,
                                    ctypes.POINTER(vp)]
    lib.bh_model_create.restype = st
    lib.bh_model_destroy.argtypes = [vp]
    lib.bh_model_destroy.restype = None
    lib.bh_set_model.argtypes = [vp, vp, vp, vp]
    lib.bh_set_model.restype = st
    lib.bh_forward.argtypes = [vp, vp, vp]
    lib.bh_forward.restype = st
    lib.bh_residual_misfit.argtypes = [vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double)]
    lib.bh_residual_misfit.restype = st
    lib.bh_adjoint_gradient.argtypes = [vp, vp, vp, vp, vp]
    lib.bh_adjoint_gradient.restype = st
    lib.bh_get_hessian.argtypes = [vp, vp, vp]
    lib.bh_get_hessian.restype = st
    lib.bh_precondition.argtypes = [vp, vp, vp, ctypes.c_double]
    lib.bh_precondition.restype = st
    lib.bh_update.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                              vp, vp]
    lib.bh_update.restype = st
    lib.bh_velocity_gradient.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.bh_velocity_gradient.restype = st
    lib.bh_get_model.argtypes = [vp, vp, vp]
    lib.bh_get_model.restype = st
    lib.bh_get_density.argtypes = [vp, vp]
    lib.bh_get_density.restype = st
    lib.bh_update_velocity.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_double), vp, vp, vp]
    lib.bh_update_velocity.restype = st
    lib.bh_profile_enable.argtypes = [vp, ctypes.c_int]
    lib.bh_profile_enable.restype = st
    lib.bh_profile_read.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_long)]
    lib.bh_profile_read.restype = st
    lib.bh_profile_reset.argtypes = [vp]
    lib.bh_profile_reset.restype = st
    lib.bh_set_option.argtypes = [vp, ctypes.c_char_p, ctypes.c_double]
    lib.bh_set_option.restype = st
    ip = ctypes.POINTER(ctypes.c_int)
    lib.bh_checkpoint_plan.argtypes = [ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, ip, ip,
                                       ctypes.c_int, ip]
    lib.bh_checkpoint_plan.restype = st
    lib.bh_plan_history.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_size_t, ip, ip, ip,
                                    ctypes.POINTER(ctypes.c_longlong)]
    lib.bh_plan_history.restype = st
    dbl = ctypes.c_double
    lib.bh_starting_model.argtypes = [ctypes.c_int, ctypes.c_int, dbl, dbl, dbl, vp, vp, vp, vp,
                                      ctypes.c_float, vp, vp, vp]
    lib.bh_starting_model.restype = st
    lib.bh_tune.argtypes = [vp, ctypes.c_int, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int]
    lib.bh_tune.restype = st
    lib.bh_tune_lookup.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ip, ip, ip, ip, ip]
    lib.bh_tune_lookup.restype = st
    lib.bh_get_info.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double)]
    lib.bh_get_info.restype = st
    lib.bh_residual_misfit_noalloc.argtypes = [vp, vp, vp, ctypes.c_size_t,
                                               ctypes.POINTER(ctypes.c_double), vp]
    lib.bh_residual_misfit_noalloc.restype = st
    lib.bh_status_string.argtypes = [st]
    lib.bh_status_string.restype = ctypes.c_char_p
    lib.bh_last_error.argtypes = [vp]
    lib.bh_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libbh takes CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _check(x, dtype, shape, name):
    if x.dtype != dtype or tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name}: expected {dtype} {tuple(shape)}, got {x.dtype} {tuple(x.shape)}")


@dataclass
class Shot:
    z_offset: int
    nz: int
    src: tuple
    rec_iz: list = field(default_factory=list)


class Model:
    """A libbh model: grid, shots, model parameters and the working state."""

    def __init__(self, nr, nz, nt, npml_r, npml_z, dr, dz, dt, f0, vp, vs, rho, shots,
                 pml_R=1e-3, stream=None, checkpoint_cap_bytes=0, snapshot_precision=0):
        self.lib = load_library()
        self.nr, self.nz, self.nt = nr, nz, nt
        self.shots = [s if isinstance(s, Shot) else Shot(s["z_offset"], s["nz"], tuple(s["src"]),
                                                         list(s["rec_iz"])) for s in shots]
        self.nshots = len(self.shots)
        self.nrec_max = max(len(s.rec_iz) for s in self.shots)
        self.device = vp.device
        for name, t in (("vp", vp), ("vs", vs), ("rho", rho)):
            _check(t, torch.float32, (nr, nz), name)
        g = GridDesc(nr, nz, nt, npml_r, npml_z, dr, dz, dt, f0, pml_R, snapshot_precision,
                     checkpoint_cap_bytes)
        self._rec = [(ctypes.c_int * max(1, len(s.rec_iz)))(*s.rec_iz) for s in self.shots]
        arr = (ShotDesc * self.nshots)()
        for k, s in enumerate(self.shots):
            arr[k] = ShotDesc(s.z_offset, s.nz, s.src[0], s.src[1], len(s.rec_iz),
                              ctypes.cast(self._rec[k], ctypes.POINTER(ctypes.c_int)))
        self.stream = stream if stream is not None else torch.cuda.current_stream(vp.device)
        h = ctypes.c_void_p()
        rc = self.lib.bh_model_create(ctypes.byref(g), nz, _ptr(vp), _ptr(vs), _ptr(rho), arr,
                                      self.nshots, ctypes.c_void_p(self.stream.cuda_stream),
                                      ctypes.byref(h))
        if rc != BH_OK:
            raise BhError(rc, self.lib.bh_last_error(None).decode())
        self.h = h

    # -- helpers
    def _rc(self, rc):
        if rc != BH_OK:
            raise BhError(rc, self.lib.bh_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.bh_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def seis_shape(self):
        return (self.nshots, self.nrec_max, self.nt)

    def empty_seis(self):
        return torch.empty(self.seis_shape(), dtype=torch.float32, device=self.device)

    # -- the C ABI, one method per entry point
    def set_model(self, vp, vs, rho):
        for name, t in (("vp", vp), ("vs", vs), ("rho", rho)):
            _check(t, torch.float32, (self.nr, self.nz), name)
        self._rc(self.lib.bh_set_model(self.h, _ptr(vp), _ptr(vs), _ptr(rho)))

    def forward(self, wavelet, seis=None):
        _check(wavelet, torch.float32, (self.nt,), "wavelet")
        seis = self.empty_seis() if seis is None else seis
        _check(seis, torch.float32, self.seis_shape(), "seis")
        self._rc(self.lib.bh_forward(self.h, _ptr(wavelet), _ptr(seis)))
        return seis

    def residual_misfit(self, seis_mod, seis_obs, resid=None):
        resid = torch.empty_like(seis_mod) if resid is None else resid
        for name, t in (("seis_mod", seis_mod), ("seis_obs", seis_obs), ("resid", resid)):
            _check(t, torch.float32, self.seis_shape(), name)
        J = ctypes.c_double()
        self._rc(self.lib.bh_residual_misfit(self.h, _ptr(seis_mod), _ptr(seis_obs), _ptr(resid),
                                             ctypes.byref(J)))
        return resid, J.value

    def adjoint_gradient(self, resid, with_rho=True, out=None):
        _check(resid, torch.float32, self.seis_shape(), "resid")
        shape = (self.nr, self.nz)
        if out is None:
            out = [torch.empty(shape, dtype=torch.float64, device=self.device)
                   for _ in range(3 if with_rho else 2)]
        g_rho = out[2] if with_rho else None
        self._rc(self.lib.bh_adjoint_gradient(self.h, _ptr(resid), _ptr(out[0]), _ptr(out[1]),
                                              _ptr(g_rho)))
        return tuple(out) if with_rho else (out[0], out[1], None)

    def hessian(self):
        H = [torch.empty((self.nr, self.nz), dtype=torch.float64, device=self.device)
             for _ in range(2)]
        self._rc(self.lib.bh_get_hessian(self.h, _ptr(H[0]), _ptr(H[1])))
        return H[0], H[1]

    def precondition(self, g_lam, g_mu, eps_rel=1e-3):
        self._rc(self.lib.bh_precondition(self.h, _ptr(g_lam), _ptr(g_mu), float(eps_rel)))
        return g_lam, g_mu

    def update(self, g_lam, g_mu, kappa=0.02, want_velocities=True):
        alpha = (ctypes.c_double * 2)()
        vp = vs = None
        if want_velocities:
            vp = torch.empty((self.nr, self.nz), dtype=torch.float32, device=self.device)
            vs = torch.empty_like(vp)
        self._rc(self.lib.bh_update(self.h, _ptr(g_lam), _ptr(g_mu), float(kappa), alpha,
                                    _ptr(vp), _ptr(vs)))
        return (alpha[0], alpha[1]), vp, vs

    def update_velocity(self, g_lam, g_mu, g_rho=None, update_rho=False, kappa=0.02,
                        want_model=True):
        """bh_update_velocity: step in (Vp, Vs) and, with update_rho, rho.
        Returns ((alpha_vp, alpha_vs, alpha_rho), vp, vs, rho)."""
        alpha = (ctypes.c_double * 3)()
        out = [None, None, None]
        if want_model:
            out = [torch.empty((self.nr, self.nz), dtype=torch.float32, device=self.device)
                   for _ in range(3)]
        self._rc(self.lib.bh_update_velocity(self.h, _ptr(g_lam), _ptr(g_mu), _ptr(g_rho),
                                             int(bool(update_rho)), float(kappa), alpha,
                                             *(_ptr(x) for x in out)))
        return (alpha[0], alpha[1], alpha[2]), out[0], out[1], out[2]

    def density(self):
        rho = torch.empty((self.nr, self.nz), dtype=torch.float32, device=self.device)
        self._rc(self.lib.bh_get_density(self.h, _ptr(rho)))
        return rho

    def tune(self, steps=32, cache_path=TUNE_CACHE):
        """bh_tune: pick the shot group size and launch form (cached per GPU
        and workload shape in cache_path, timed on a miss).  Returns the
        library's description of the choice."""
        buf = ctypes.create_string_buffer(8192)
        path = cache_path.encode() if cache_path else None
        self._rc(self.lib.bh_tune(self.h, int(steps), path, buf, len(buf)))
        return buf.value.decode()

    def set_option(self, key, value):
        """bh_set_option: "persistent", "group", "tile_code", "split",
        "tile_order", "pipe_grid", "barrier_timeout_ms", "barrier_extra_arrivals"."""
        self._rc(self.lib.bh_set_option(self.h, key.encode(), float(value)))

    def info(self, key):
        """bh_get_info: history_steps, snapshots, recompute_steps, tiles, ..."""
        v = ctypes.c_double()
        self._rc(self.lib.bh_get_info(self.h, key.encode(), ctypes.byref(v)))
        return v.value

    def profile(self, every):
        """Sample kernel timing on every every-th step (0 = off)."""
        self._rc(self.lib.bh_profile_enable(self.h, int(every)))

    def profile_read(self):
        """{kernel name: (total ms, sampled launches)} since the last reset."""
        out = {}
        for k, name in enumerate(KERNELS):
            t, n = ctypes.c_double(), ctypes.c_long()
            self._rc(self.lib.bh_profile_read(self.h, k, ctypes.byref(t), ctypes.byref(n)))
            out[name] = (t.value, n.value)
        return out

    def profile_reset(self):
        self._rc(self.lib.bh_profile_reset(self.h))

    def velocity_gradient(self, g_lam, g_mu, g_rho=None):
        """bh_velocity_gradient: (g_vp, g_vs, g_rho at fixed velocities), float32."""
        shape = (self.nr, self.nz)
        out = [torch.empty(shape, dtype=torch.float32, device=self.device) for _ in range(3)]
        self._rc(self.lib.bh_velocity_gradient(self.h, _ptr(g_lam), _ptr(g_mu), _ptr(g_rho),
                                               _ptr(out[0]), _ptr(out[1]), _ptr(out[2])))
        return tuple(out)

    def velocities(self):
        vp = torch.empty((self.nr, self.nz), dtype=torch.float32, device=self.device)
        vs = torch.empty_like(vp)
        self._rc(self.lib.bh_get_model(self.h, _ptr(vp), _ptr(vs)))
        return vp, vs


def model_from_workload(w, device="cuda", **kw):
    """Build a Model from a synthetic.Workload (start model)."""
    t = lambda a: torch.from_numpy(a).to(device)
    return Model(w.nr, w.nz, w.nt, w.npml_r, w.npml_z, w.dr, w.dz, w.dt, w.f0, t(w.vp), t(w.vs),
                 t(w.rho), w.shots, pml_R=w.pml_R, **kw)


def residual_misfit_noalloc(seis_mod, seis_obs, resid, stream=None):
    """bh_residual_misfit_noalloc: Eq. 5 residual into `resid` and the Eq. 1
    misfit J, with no device allocation by the library (and none here: the
    caller passes every buffer).  Returns J."""
    lib = load_library()
    for name, t in (("seis_obs", seis_obs), ("resid", resid)):
        if t.dtype != torch.float32 or t.numel() != seis_mod.numel():
            raise ValueError(f"{name}: float32 tensor with {seis_mod.numel()} elements expected")
    stream = stream if stream is not None else torch.cuda.current_stream(seis_mod.device)
    J = ctypes.c_double()
    rc = lib.bh_residual_misfit_noalloc(_ptr(seis_mod), _ptr(seis_obs), _ptr(resid),
                                        seis_mod.numel(), ctypes.byref(J),
                                        ctypes.c_void_p(stream.cuda_stream))
    if rc != BH_OK:
        raise BhError(rc, lib.bh_last_error(None).decode())
    return J.value


def checkpoint_plan(nseg, nsnap):
    """bh_checkpoint_plan (host only): (spine [(segment, slot)], actions [(kind, a, b)])."""
    lib = load_library()
    na, ns = ctypes.c_int(), ctypes.c_int()
    cap_a, cap_s = 4 * nseg * (nsnap + 2) + 16, nseg + 1
    while True:
        acts = (ctypes.c_int * (3 * cap_a))()
        sp = (ctypes.c_int * (2 * cap_s))()
        rc = lib.bh_checkpoint_plan(nseg, nsnap, acts, cap_a, ctypes.byref(na), sp, cap_s,
                                    ctypes.byref(ns))
        if rc == BH_OK:
            break
        if na.value <= cap_a and ns.value <= cap_s:
            raise BhError(rc, lib.bh_last_error(None).decode())
        cap_a, cap_s = max(cap_a, na.value), max(cap_s, ns.value)
    spine = [(sp[2 * k], sp[2 * k + 1]) for k in range(ns.value)]
    actions = [(acts[3 * k], acts[3 * k + 1], acts[3 * k + 2]) for k in range(na.value)]
    return spine, actions


def plan_history(nt, hist_step_bytes, snapshot_bytes, cap_bytes):
    """bh_plan_history (host only): (L, nsnap, tail, recomputed steps) of the
    forward-history plan under a byte cap."""
    lib = load_library()
    L, s, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc_ = ctypes.c_longlong()
    rc = lib.bh_plan_history(int(nt), float(hist_step_bytes), float(snapshot_bytes),
                             int(cap_bytes), ctypes.byref(L), ctypes.byref(s), ctypes.byref(t),
                             ctypes.byref(rc_))
    if rc != BH_OK:
        raise BhError(rc, lib.bh_last_error(None).decode())
    return L.value, s.value, t.value, rc_.value


def starting_model(nr, dr, r_wall, r_far, vp_wall, vs_wall, vp_far, vs_far, vp_fluid=1500.0,
                   stream=None):
    """bh_starting_model: (vp, vs) [nr, nz] float32 CUDA tensors from the
    velocity logs at the wall and at r_far ([nz] float32 CUDA tensors)."""
    lib = load_library()
    nz = vp_wall.numel()
    for name, t in (("vp_wall", vp_wall), ("vs_wall", vs_wall), ("vp_far", vp_far),
                    ("vs_far", vs_far)):
        _check(t, torch.float32, (nz,), name)
    vp = torch.empty((nr, nz), dtype=torch.float32, device=vp_wall.device)
    vs = torch.empty_like(vp)
    stream = stream if stream is not None else torch.cuda.current_stream(vp_wall.device)
    rc = lib.bh_starting_model(int(nr), int(nz), float(dr), float(r_wall), float(r_far),
                               _ptr(vp_wall), _ptr(vs_wall), _ptr(vp_far), _ptr(vs_far),
                               float(vp_fluid), _ptr(vp), _ptr(vs),
                               ctypes.c_void_p(stream.cuda_stream))
    if rc != BH_OK:
        raise BhError(rc, lib.bh_last_error(None).decode())
    return vp, vs


def tune_lookup(cache_path, gpu_name, nr, window_pitch, nshots):
    """bh_tune_lookup (host only): (group, form, tile code, split, tile
    order) cached for the key, or None."""
    lib = load_library()
    g, f, v, sp, od = (ctypes.c_int() for _ in range(5))
    rc = lib.bh_tune_lookup(cache_path.encode(), gpu_name.encode(), int(nr), int(window_pitch),
                            int(nshots), ctypes.byref(g), ctypes.byref(f), ctypes.byref(v),
                            ctypes.byref(sp), ctypes.byref(od))
    if rc == 6:
        return None
    if rc != BH_OK:
        raise BhError(rc, lib.bh_last_error(None).decode())
    return g.value, f.value, v.value, sp.value, od.value
