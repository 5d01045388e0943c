"""Synthetic borehole logging workloads (models, shots, wavelet), seeded.

The paper inverts synthetic data only (Numerical Examples) and prints no
model values, so the workloads below stand in for its layered and
flushed-zone models: a fluid-filled borehole of radius 0.10 m (water,
Vp 1500 m/s, rho 1000 kg/m^3) in an axially layered formation with a radial
damage annulus, a monopole source and pressure receivers on the axis
(Numerical Examples; Fig. 2, Fig. 3).

Every array is float32 (the precision the CUDA path steps in); the oracle
upcasts the same values to float64.  Indices are window coordinates: cell
(i, j) sits at r = (i + 1/2) dr, z = j dz.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FLUID_VP = 1500.0
FLUID_RHO = 1000.0
BOREHOLE_RADIUS = 0.10


@dataclass
class Workload:
    name: str
    nr: int
    nz: int                # global model length in cells
    nt: int
    npml_r: int
    npml_z: int
    dr: float
    dz: float
    dt: float
    f0: float
    vp: np.ndarray         # [nr, nz] float32, start model
    vs: np.ndarray
    rho: np.ndarray
    vp_true: np.ndarray    # [nr, nz] float32, model that makes the "measured" data
    vs_true: np.ndarray
    rho_true: np.ndarray
    shots: list = field(default_factory=list)  # dicts: z_offset, nz, src, rec_iz
    wavelet: np.ndarray | None = None          # [nt] float32, s(t_{n+1/2})
    pml_R: float = 1e-3
    logs: dict | None = None                   # velocity logs at the wall and 1 m beyond

    @property
    def nshots(self):
        return len(self.shots)

    @property
    def nrec(self):
        return max(len(s["rec_iz"]) for s in self.shots)

    def cell_steps(self):
        """Cell updates of one forward pass over all shots."""
        return sum(self.nr * s["nz"] * self.nt for s in self.shots)


def ricker(nt: int, dt: float, f0: float, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet of unit amplitude sampled at t = (n + 1/2) dt, with
    delay t0 = 1.5 / f0 (the paper names no wavelet; this is the reading)."""
    t0 = 1.5 / f0 if t0 is None else t0
    t = (np.arange(nt) + 0.5) * dt - t0
    a = (np.pi * f0 * t) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


def _borehole(nr, nz, dr, fluid_radius=BOREHOLE_RADIUS):
    """Boolean [nr] of radial cells inside the borehole fluid."""
    r = (np.arange(nr) + 0.5) * dr
    return r < fluid_radius


def _fill_fluid(vp, vs, rho, fluid_rows):
    vp[fluid_rows, :] = FLUID_VP
    vs[fluid_rows, :] = 0.0
    rho[fluid_rows, :] = FLUID_RHO


def _f32(*arrs):
    return [np.ascontiguousarray(a, dtype=np.float32) for a in arrs]


def homogeneous(nr, nz, nt, npml_r, npml_z, h, dt, f0, vp, vs, rho, src, rec_iz,
                name="homogeneous"):
    """A homogeneous whole space (vs = 0 gives a fluid), single shot."""
    a = np.full((nr, nz), vp)
    b = np.full((nr, nz), vs)
    c = np.full((nr, nz), rho)
    a, b, c = _f32(a, b, c)
    return Workload(name, nr, nz, nt, npml_r, npml_z, h, h, dt, f0, a, b, c, a.copy(),
                    b.copy(), c.copy(),
                    [dict(z_offset=0, nz=nz, src=tuple(src), rec_iz=list(rec_iz))],
                    ricker(nt, dt, f0))


def config0():
    """Single-shot correctness case: nr 80 (20-cell C-PML), nz 400 (20-cell
    C-PML top and bottom), 1 cm cells, dt 1 us, 2500 steps, 5 kHz Ricker on
    the axis at z = 0.4 m, 8 receivers on the axis at 2.00 ... 3.05 m.
    Formation Vp 4000, Vs 2300, rho 2500; the true model adds a damaged
    annulus at r = 0.10 ... 0.20 m with Vp and Vs lowered by 10 %."""
    nr, nz, h, dt, nt = 80, 400, 0.01, 1e-6, 2500
    vp = np.full((nr, nz), 4000.0)
    vs = np.full((nr, nz), 2300.0)
    rho = np.full((nr, nz), 2500.0)
    fl = _borehole(nr, nz, h)
    _fill_fluid(vp, vs, rho, fl)
    vpt, vst = vp.copy(), vs.copy()
    r = (np.arange(nr) + 0.5) * h
    ann = (r >= 0.10) & (r < 0.20)
    vpt[ann, :] *= 0.9
    vst[ann, :] *= 0.9
    vp, vs, rho, vpt, vst = _f32(vp, vs, rho, vpt, vst)
    rec = [int(round(z / h)) for z in np.arange(8) * 0.15 + 2.00]
    shot = dict(z_offset=0, nz=nz, src=(0, int(round(0.4 / h))), rec_iz=rec)
    return Workload("c0", nr, nz, nt, 20, 20, h, h, dt, 5e3, vp, vs, rho, vpt, vst,
                    rho.copy(), [shot], ricker(nt, dt, 5e3))


def _layered(rng, nr, nz, h, fluid_rows):
    """Axially layered formation: beds 0.3-1.0 m thick, Vp U(3000, 5000),
    Vs = Vp / U(1.7, 1.9), rho U(2200, 2600); plus one radial damage zone of
    depth U(0.05, 0.25) m beyond the borehole wall with Vp and Vs lowered by
    U(5, 15) %.  Returns start (undamaged) and true (damaged) models."""
    vp = np.empty((nr, nz))
    vs = np.empty((nr, nz))
    rho = np.empty((nr, nz))
    z = 0
    while z < nz:
        thick = max(1, int(round(rng.uniform(0.3, 1.0) / h)))
        bvp = rng.uniform(3000.0, 5000.0)
        vp[:, z: z + thick] = bvp
        vs[:, z: z + thick] = bvp / rng.uniform(1.7, 1.9)
        rho[:, z: z + thick] = rng.uniform(2200.0, 2600.0)
        z += thick
    _fill_fluid(vp, vs, rho, fluid_rows)
    depth = rng.uniform(0.05, 0.25)
    drop = rng.uniform(0.05, 0.15)
    r = (np.arange(nr) + 0.5) * h
    dmg = (r >= BOREHOLE_RADIUS) & (r < BOREHOLE_RADIUS + depth)
    vpt, vst = vp.copy(), vs.copy()
    vpt[dmg, :] *= 1.0 - drop
    vst[dmg, :] *= 1.0 - drop
    return vp, vs, rho, vpt, vst


def _shot(z_offset, nz, npml_z, h):
    """Source on the axis 80 cells below the window's top C-PML; 13
    receivers on the axis at offsets 3.00 ... 4.80 m (0.15 m apart)."""
    src_iz = npml_z + 80
    rec = [src_iz + int(round(o / h)) for o in 3.0 + 0.15 * np.arange(13)]
    assert rec[-1] < nz - npml_z, "receivers must sit above the bottom C-PML"
    return dict(z_offset=int(z_offset), nz=int(nz), src=(0, src_iz), rec_iz=rec)


def config1(seed=0):
    """Production single shot: nr 240 (40-cell C-PML), nz 1600 (40-cell
    C-PML), 5 mm cells, dt 0.5 us, 8000 steps, 10 kHz Ricker."""
    rng = np.random.default_rng(seed)
    nr, nz, h, dt, nt, npml = 240, 1600, 0.005, 0.5e-6, 8000, 40
    vp, vs, rho, vpt, vst = _layered(rng, nr, nz, h, _borehole(nr, nz, h))
    vp, vs, rho, vpt, vst = _f32(vp, vs, rho, vpt, vst)
    return Workload("c1", nr, nz, nt, npml, npml, h, h, dt, 1e4, vp, vs, rho, vpt, vst,
                    rho.copy(), [_shot(0, nz, npml, h)], ricker(nt, dt, 1e4))


def _batched(name, rng, nshots, nz_lo, nz_hi, model_len_cells, nt=8000):
    nr, h, dt, npml = 240, 0.005, 0.5e-6, 40
    vp, vs, rho, vpt, vst = _layered(rng, nr, model_len_cells, h, _borehole(nr, 0, h))
    vp, vs, rho, vpt, vst = _f32(vp, vs, rho, vpt, vst)
    step = int(round(0.15 / h))
    shots = []
    for s in range(nshots):
        nzs = int(rng.integers(nz_lo, nz_hi + 1))
        z0 = s * step
        assert z0 + nzs <= model_len_cells
        shots.append(_shot(z0, nzs, npml, h))
    return Workload(name, nr, model_len_cells, nt, npml, npml, h, h, dt, 1e4, vp, vs, rho,
                    vpt, vst, rho.copy(), shots, ricker(nt, dt, 1e4))


def config2(seed=0, nt=8000):
    """Batched logging run: 64 shots, source stepped 0.15 m, windows
    nz ~ U{1400..2000} cells over a 20 m layered model."""
    return _batched("c2", np.random.default_rng(seed), 64, 1400, 2000, 4000, nt)


def config3(seed=0, nt=12000):
    """Large single shot: nr 400, nz 4000, 5 mm cells, 12000 steps."""
    rng = np.random.default_rng(seed)
    nr, nz, h, dt, npml = 400, 4000, 0.005, 0.5e-6, 40
    vp, vs, rho, vpt, vst = _layered(rng, nr, nz, h, _borehole(nr, nz, h))
    vp, vs, rho, vpt, vst = _f32(vp, vs, rho, vpt, vst)
    return Workload("c3", nr, nz, nt, npml, npml, h, h, dt, 1e4, vp, vs, rho, vpt, vst,
                    rho.copy(), [_shot(0, nz, npml, h)], ricker(nt, dt, 1e4))


def config4(seed=0, nt=8000):
    """256 shots with windows nz ~ U{1200..2400} over a layered model
    extended to 256 * 0.15 m + 2400 cells + 1 m (about 51.4 m)."""
    length = 256 * 30 + 2400 + 200
    return _batched("c4", np.random.default_rng(seed), 256, 1200, 2400, length, nt)


def tiny_borehole(seed=0, nr=24, nz=48, npml=6, nt=300, h=0.01, dt=1e-6, f0=15e3,
                  fluid_rows=4, nrec=3, heterogeneous=True):
    """A small borehole model for finite-difference gradient and dot-product
    tests: fluid in the first `fluid_rows` radial cells, a formation with
    random per-cell perturbations (so that every cell matters)."""
    rng = np.random.default_rng(seed)
    vp = np.full((nr, nz), 3500.0)
    vs = np.full((nr, nz), 2000.0)
    rho = np.full((nr, nz), 2400.0)
    if heterogeneous:
        vp *= 1.0 + 0.05 * rng.standard_normal((nr, nz))
        vs *= 1.0 + 0.05 * rng.standard_normal((nr, nz))
        rho *= 1.0 + 0.05 * rng.standard_normal((nr, nz))
    vp[:fluid_rows] = FLUID_VP
    vs[:fluid_rows] = 0.0
    rho[:fluid_rows] = FLUID_RHO
    vpt = vp * (1.0 + 0.03 * rng.standard_normal((nr, nz)))
    vst = vs * (1.0 + 0.03 * rng.standard_normal((nr, nz)))
    vpt[:fluid_rows], vst[:fluid_rows] = vp[:fluid_rows], vs[:fluid_rows]
    vp, vs, rho, vpt, vst = _f32(vp, vs, rho, vpt, vst)
    src = (0, npml + 3)
    rec = list(np.linspace(npml + 10, nz - npml - 2, nrec).round().astype(int))
    shot = dict(z_offset=0, nz=nz, src=src, rec_iz=[int(x) for x in rec])
    return Workload("tiny", nr, nz, nt, npml, npml, h, h, dt, f0, vp, vs, rho, vpt, vst,
                    rho.copy(), [shot], ricker(nt, dt, f0))





# ---------------------------------------------------------------------------
# Multi-source logging tool (Numerical Examples, Fig. 2): thirteen receiver
# stations 0.5 ft apart above three monopoles (lower-near, far, ultra-far);
# the tool logs every 0.5 ft.  The paper realigns the records of the three
# sources to one source and thirty-nine receivers.  Reading (the paper prints
# no source offsets): the far and ultra-far monopoles sit 13 and 26 stations
# (6.5 ft and 13 ft) below the lower-near one, so the three arrays, seen from
# one source depth, cover 39 consecutive stations; the lower-near source is
# `near_offset` below the first receiver.

FT = 0.3048
STATION = 0.5 * FT
TOOL_SOURCES = ("lower-near", "far", "ultra-far")
TOOL_STATIONS = 13


def tool_records(ndepths: int, z_first: float, near_offset: float = 3.0,
                 step: float = STATION, spacing: float = STATION):
    """The raw acquisition table of a logging run: one record per (tool
    depth, monopole): source depth and the depths of the 13 receivers.  The
    tool moves `step` per depth; z grows downwards and the receivers sit
    above the sources (smaller z).  z_first: depth of the lower-near source
    at the first tool depth."""
    recs = []
    for d in range(ndepths):
        z_near = z_first + d * step
        for k, name in enumerate(TOOL_SOURCES):
            zs = z_near + k * TOOL_STATIONS * spacing
            rz = [z_near - near_offset - q * spacing for q in range(TOOL_STATIONS)]
            recs.append(dict(depth=d, source=name, z_src=zs, z_rec=rz))
    return recs


def realign(recs, spacing: float = STATION, tol: float = 1e-9):
    """Realigned gathers: records whose sources sit at the same depth merge
    into one gather of one source and the union of their receivers, ordered
    by offset.  Returns {source depth: [(offset, record index, receiver
    index), ...]} for the source depths that all three monopoles visit."""
    by_src = {}
    for i, r in enumerate(recs):
        key = round(r["z_src"] / spacing)
        by_src.setdefault(key, []).append(i)
    out = {}
    for key, idx in by_src.items():
        if len(idx) != len(TOOL_SOURCES):
            continue
        zs = recs[idx[0]]["z_src"]
        rows = []
        for i in idx:
            assert abs(recs[i]["z_src"] - zs) < tol
            for q, zr in enumerate(recs[i]["z_rec"]):
                rows.append((zs - zr, i, q))
        out[zs] = sorted(rows)
    return out


def tool_logging_run(seed=0, ndepths=16, nt=6000, near_offset=3.0, h=0.005, dt=0.5e-6,
                     f0=1e4, npml=40, nr=240, margin=0.5, name="tool"):
    """Batched workload of the realigned tool geometry: one shot per source
    depth that all three monopoles visit, each with its 39 receivers on the
    axis, its own window (margin above the farthest receiver and below the
    source) of a layered model with a damaged annulus like the production
    shot's."""
    rng = np.random.default_rng(seed)
    recs_probe = tool_records(1, 0.0, near_offset)
    span = near_offset + (3 * TOOL_STATIONS - 1) * STATION  # source to farthest receiver
    top = npml * h + margin
    # every source depth realigned needs 2 * 13 further tool depths
    ndep_raw = ndepths + 2 * TOOL_STATIONS
    z_first = top + span
    recs = tool_records(ndep_raw, z_first, near_offset)
    gathers = realign(recs)
    zs_sorted = sorted(gathers)[:ndepths]
    length_m = zs_sorted[-1] + margin + npml * h
    nzg = int(np.ceil(length_m / h)) + 1
    vp, vs, rho, vpt, vst = _layered(rng, nr, nzg, h, _borehole(nr, 0, h))
    vp, vs, rho, vpt, vst = _f32(vp, vs, rho, vpt, vst)
    shots = []
    for zs in zs_sorted:
        rows = gathers[zs]
        z_top_rec = zs - max(o for o, _, _ in rows)
        z0 = int(np.floor((z_top_rec - margin) / h)) - npml
        z1 = int(np.ceil((zs + margin) / h)) + npml
        z0 = max(z0, 0)
        z1 = min(z1, nzg)
        src_iz = int(round(zs / h)) - z0
        rec_iz = [int(round((zs - o) / h)) - z0 for o, _, _ in rows]
        shots.append(dict(z_offset=z0, nz=z1 - z0, src=(0, src_iz), rec_iz=sorted(rec_iz)))
    del recs_probe
    return Workload(name, nr, nzg, nt, npml, npml, h, h, dt, f0, vp, vs, rho, vpt, vst,
                    rho.copy(), shots, ricker(nt, dt, f0))


def flushed_zone(seed=0, nshots=8, nt=8000, h=0.005, dt=0.5e-6, f0=1e4, npml=40, nr=240,
                 nz_window=1700, name="flushed"):
    """A layered formation with a low-velocity flushed (invaded) zone around
    the borehole whose depth changes from bed to bed: velocity variation in
    both the radial and the axial direction, like the paper's second model
    (Numerical Examples, Fig. 7; its values are not printed).  Beds 0.3-1.0 m
    thick as in the production shot; in each bed the flushed zone reaches
    U(0.05, 0.35) m beyond the wall with Vp lowered by U(8, 15) % and Vs by
    half as much.  The true model has the flushed zone, the start model is the
    virgin formation.  `logs` holds what the near- and far-offset data see at
    every depth: the velocities at the wall and one meter beyond it.  Shots
    step 0.15 m with windows of nz_window cells, geometry as the production
    shot."""
    rng = np.random.default_rng(seed)
    step = int(round(0.15 / h))
    nzg = (nshots - 1) * step + nz_window
    fluid = _borehole(nr, 0, h)
    vp = np.empty((nr, nzg))
    vs = np.empty((nr, nzg))
    rho = np.empty((nr, nzg))
    vpt = np.empty((nr, nzg))
    vst = np.empty((nr, nzg))
    r = (np.arange(nr) + 0.5) * h
    z = 0
    while z < nzg:
        thick = max(1, int(round(rng.uniform(0.3, 1.0) / h)))
        bvp = rng.uniform(3000.0, 5000.0)
        bvs = bvp / rng.uniform(1.7, 1.9)
        brho = rng.uniform(2200.0, 2600.0)
        depth = rng.uniform(0.05, 0.35)
        drop = rng.uniform(0.08, 0.15)
        sl = np.s_[:, z: z + thick]
        vp[sl], vs[sl], rho[sl] = bvp, bvs, brho
        inv = (r >= BOREHOLE_RADIUS) & (r < BOREHOLE_RADIUS + depth)
        vpt[sl] = bvp
        vst[sl] = bvs
        vpt[inv, z: z + thick] = bvp * (1.0 - drop)
        vst[inv, z: z + thick] = bvs * (1.0 - drop / 2)
        z += thick
    _fill_fluid(vp, vs, rho, fluid)
    vpt[fluid], vst[fluid] = vp[fluid], vs[fluid]
    vp, vs, rho, vpt, vst = _f32(vp, vs, rho, vpt, vst)
    shots = [_shot(s * step, nz_window, npml, h) for s in range(nshots)]
    w = Workload(name, nr, nzg, nt, npml, npml, h, h, dt, f0, vp, vs, rho, vpt, vst,
                 rho.copy(), shots, ricker(nt, dt, f0))
    i_wall = int(np.argmax(~fluid))
    i_far = int(np.argmin(np.abs(r - (BOREHOLE_RADIUS + 1.0))))
    w.logs = dict(r_wall=BOREHOLE_RADIUS, r_far=BOREHOLE_RADIUS + 1.0,
                  vp_wall=np.ascontiguousarray(vpt[i_wall]), vs_wall=np.ascontiguousarray(vst[i_wall]),
                  vp_far=np.ascontiguousarray(vpt[min(i_far, nr - npml - 1)]),
                  vs_far=np.ascontiguousarray(vst[min(i_far, nr - npml - 1)]))
    return w


PRESETS = {"c0": config0, "c1": config1, "c2": config2, "c3": config3, "c4": config4,
           "flushed": flushed_zone, "tool": tool_logging_run}
