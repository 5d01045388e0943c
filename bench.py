#!/usr/bin/env python
"""Benchmark of the borehole FWI hot path on GB300.

One step = one full inversion iteration of the batched logging run (64
shots stepped 0.15 m along a 20 m layered model, windows of 1400-2000 cells
by 240, 8000 steps, 10 kHz): forward modelling of every shot, residual and
misfit, adjoint modelling with the fused gradient correlation, per-cell
gradients summed over the shots, preconditioner, and model update, all
through the C ABI of libbh.  The density is known (the paper takes it from
logs), so the iteration asks for the lambda and mu gradients only.  The
single production shot (240 x 1600, 8000 steps) is timed after it as a
secondary line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                  [--config c0..c4] [--cap-gb GB] [--snap fp32|bf16|fp16]

Prints one JSON line (rank 0).  With N > 1 (launched by torchrun) every rank
inverts its own independent workload (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s and gradient evals/s (fwd+adj+grad) at 1 GB300; % of HBM roofline"
UNIT = "Gcell-updates/s"
PROFILE_EVERY = 64
CPU_SAMPLE_STEPS = 150
REF_SAMPLE_STEPS = 100
L2_BYTES = 129e6
# checkpoint byte cap per workload when --cap-gb is not given (0: every step
# of the forward history stored)
DEFAULT_CAP_GB = {"c0": 0.0, "c1": 0.0, "c2": 240.0, "c3": 4.0, "c4": 240.0, "flushed": 100.0,
                  "tool": 150.0}
DEFAULT_SNAP = {"c4": "bf16"}
E2E_STEPS = 3
SECONDARY_STEPS = 10

# Algorithmic bytes per cell and step of each stepping kernel, from the FP32
# byte model of the method: each of the six wavefields read and written once
# per step (the velocity half-step owns v_r, v_z, the stress half-step the
# four stresses); lambda, mu, rho read once per step (the stress half-step
# reads lambda and mu, the velocity half-step rho), not counted when several
# shots share one model (it then stays in L2); the C-PML memories read and
# written in their strips only (s = npml_r / nr + 2 npml_z / nz of the
# window; 16 s per half-step); the forward history v_r, v_z written by the
# forward stress half-step of a stored step and read once by the adjoint;
# the three gradient accumulators G_lambda, G_mu,nn, G_mu,rz read and
# written.  Kahan compensation, the pseudo-Hessian and the density
# correlation are not counted (implementation extras).
def method_bytes_per_cell(kernel: str, s: float, shared_model: bool, hist: float = 1.0) -> float:
    m = 0.0 if shared_model else 1.0
    return {
        "fwd_vel": 16 + 4 * m + 16 * s,
        "fwd_stress": 32 + 8 * m + 8 * hist + 16 * s,
        "adj_stress": 16 + 8 * m + 8 + 24 + 16 * s,
        "adj_vel": 32 + 4 * m + 16 * s,
    }[kernel]


# Every array a launch of this implementation touches, once per cell and
# step (FP32 fields, per-window coefficient planes, Kahan pairs, pseudo-
# Hessian, both history planes the adjoint reads): the traffic the kernels
# would move with no cache reuse at all.
def all_array_bytes_per_cell(kernel: str, s: float, with_rho: bool, hist: float = 1.0) -> float:
    return {
        # 4 stresses read, v_r v_z read+write, 2 buoyancies, 4 memories r+w
        "fwd_vel": 16 + 16 + 8 + 16 * s,
        # v_r v_z read, 4 stresses read+write, lambda mu mu_h, history write, 4 memories
        "fwd_stress": 8 + 32 + 12 + 8 * hist + 16 * s,
        # 4 adjoint stresses read, 2 adjoint velocities r+w, lambda mu mu_h,
        # history v^{n+1/2} (and v^{n-1/2} for rho), 3 (5) Kahan pairs r+w,
        # 3 Hessian r+w, 4 adjoint memories (read one bank, write the other)
        "adj_stress": 16 + 16 + 12 + 8 + 48 + 24 + 16 * s + (8 + 32 if with_rho else 0),
        # 2 adjoint velocities read, 4 adjoint stresses r+w, 2 buoyancies, 4 memories
        "adj_vel": 8 + 32 + 8 + 16 * s,
        # a fused forward step: the six fields read and written once, five
        # coefficients, history write, 8 memories r+w in their strips
        "fwd_step": 48 + 20 + 8 * hist + 32 * s,
    }[kernel]


# persistent kernels run both half-steps of every time step of a shot group
PERSIST_PARTS = {"fwd_persist": ("fwd_vel", "fwd_stress"), "adj_persist": ("adj_stress", "adj_vel"),
                 "fwd_step": ("fwd_vel", "fwd_stress"),
                 "fwd_vel": ("fwd_vel",), "fwd_stress": ("fwd_stress",),
                 "adj_stress": ("adj_stress",), "adj_vel": ("adj_vel",)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_sha():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2005_00281_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per cell and step of a kernel from a committed ncu summary
    (profiles/traffic_<kernel>_<workload>.txt), if it was taken on the
    current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", f"traffic_{kernel}_{workload}.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    with open(p) as f:
        for line in f:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("source_sha") != source_sha():
        return None
    try:
        return float(vals["dram_bytes_per_cell_step"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_config(w, nt=None):
    if w.nshots > 1:
        shots = (f"{w.nshots} shots, windows nz {min(s['nz'] for s in w.shots)}-"
                 f"{max(s['nz'] for s in w.shots)} of a {w.nz}-cell model")
    elif w.shots[0]["nz"] != w.nz:
        shots = f"single shot, window nz {w.shots[0]['nz']} of a {w.nz}-cell model"
    else:
        shots = f"single shot, nz {w.nz}"
    return {"workload": f"{w.name}: borehole FWI iteration, {shots}, nr {w.nr} "
                        f"(C-PML {w.npml_r}/{w.npml_z}), {nt or w.nt} steps, "
                        f"h {w.dr} m, dt {w.dt} s, f0 {w.f0:g} Hz, {w.nrec} receivers",
            "nr": w.nr, "nz": w.nz, "nt": nt or w.nt, "nshots": w.nshots,
            "l2": "inputs larger than L2: the forward history streamed every step is "
                  f"{2 * 8 * w.cell_steps() * (nt or w.nt) / w.nt / 1e9:.1f} GB (write + read)"}


# ---------------------------------------------------------------- oracle

def oracle_sample(w, nt_sample):
    """The FP64 oracle as it stands, one forward + adjoint + gradient of the
    workload's first shot truncated to nt_sample steps.  Returns
    (Gcell-updates/s, seconds, threads)."""
    import numpy as np
    from oracle import oracle as O

    sh = w.shots[0]
    g = O.Grid(w.nr, sh["nz"], nt_sample, w.npml_r, w.npml_z, w.dr, w.dz, w.dt, w.f0, w.pml_R)
    z0 = sh["z_offset"]
    sl = np.s_[:, z0: z0 + sh["nz"]]
    vp, vs, rho = (np.ascontiguousarray(a[sl]) for a in (w.vp, w.vs, w.rho))
    wav = w.wavelet[:nt_sample]
    t0 = time.perf_counter()
    seis, vh = O.forward(g, vp, vs, rho, wav, sh["src"], sh["rec_iz"])
    resid, J = O.residual_misfit(seis, np.zeros_like(seis))
    acc, _, _ = O.adjoint(g, vp, vs, rho, resid, sh["src"], sh["rec_iz"], vh)
    O.finalize(g, vp, vs, rho, acc)
    dt = time.perf_counter() - t0
    cells = 2.0 * w.nr * sh["nz"] * nt_sample
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return cells / dt / 1e9, dt, threads


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals = []
    for k in range(args.warmup + args.steps):
        v, sec, threads = oracle_sample(w, REF_SAMPLE_STEPS)
        if k >= args.warmup:
            vals.append((v, sec))
    value = statistics.mean(v for v, _ in vals)
    sample = (f"first shot of {w.name}, nt truncated to {REF_SAMPLE_STEPS} of {w.nt} steps "
              f"(forward + adjoint + gradient); forward loops OpenMP, adjoint serial")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(s for _, s in vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, REF_SAMPLE_STEPS),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------- multi-rank host logic
#
# With N > 1 every rank inverts its own independent shot of the same sizes
# (seed = rank): the path shards by shots with no data-path collective.  The
# barrier and the max over ranks serve the timing only; the job's value is
# the cells of all ranks over the slowest rank's time.

def rank_workload(config: str, rank: int):
    """The workload rank `rank` inverts: the named preset, seeded by rank."""
    from synthetic import PRESETS
    return PRESETS[config](seed=rank)


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over the ranks of the default process group."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    tt = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(cells_per_rank: float, world: int, ms: float) -> float:
    """Whole-job Gcell-updates/s: every rank's cells over the max-over-ranks time."""
    return world * cells_per_rank / (ms / 1e3) / 1e9


# ---------------------------------------------------------------- GPU arm

def shot_pml_fraction(w):
    """Cell-weighted s = npml_r / nr + 2 npml_z / nz over the shot windows."""
    cells = [w.nr * sh["nz"] for sh in w.shots]
    ss = [w.npml_r / w.nr + 2.0 * w.npml_z / sh["nz"] for sh in w.shots]
    return sum(c * x for c, x in zip(cells, ss)) / sum(cells)


def state_bytes_per_group(w, group=32):
    """Bytes of window state one shot group's launch touches: 6 fields and
    the C-PML memories (strips) of the forward and adjoint, the per-window
    coefficient planes, the Kahan pairs and pseudo-Hessian planes."""
    P = (max(sh["nz"] for sh in w.shots) + 31) // 32 * 32
    plane = w.nr * P * 4
    s = shot_pml_fraction(w)
    planes = 6 + 8 * s + 6 + 16 * s + 13 + 5
    return min(group, w.nshots) * planes * plane


def measure(w, args, dev, world, rank, steps, warmup, cap, prec, with_rho, e2e_steps,
            label):
    """Time `steps` inversion iterations of workload w through the C ABI
    (after `warmup`), then `e2e_steps` with host inputs; returns the JSON
    fields of one bench line."""
    import ctypes
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2005_00281_gb300.bh import TUNE_CACHE, model_from_workload

    local = dev.index
    stream = torch.cuda.current_stream(dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    # observed data: forward modelling in the true model (outside the timing)
    true = model_from_workload(w, device=dev, checkpoint_cap_bytes=cap)
    true.set_model(t(w.vp_true), t(w.vs_true), t(w.rho_true))
    wav = t(w.wavelet)
    obs = true.forward(wav).clone()
    torch.cuda.synchronize()
    true.close()
    del true

    m = model_from_workload(w, device=dev, checkpoint_cap_bytes=cap, snapshot_precision=prec)
    tuning = None
    if args.per_step:
        m.set_option("persistent", 0)
    elif args.persistent:
        m.set_option("persistent", 1)
    elif not args.no_tune:
        # launch configuration from the autotuner (cached per GPU and shape)
        tuning = m.tune(steps=64, cache_path=args.tune_cache or TUNE_CACHE)
    for kv in args.opt or []:
        key, val = kv.split("=")
        m.set_option(key, float(val))
    start_model = (t(w.vp), t(w.vs), t(w.rho))
    seis = m.empty_seis()
    resid = torch.empty_like(seis)
    shape = (w.nr, w.nz)
    g = [torch.empty(shape, dtype=torch.float64, device=dev) for _ in range(3)]
    g_rho = g[2] if with_rho else None
    vp_out = torch.empty(shape, dtype=torch.float32, device=dev)
    vs_out = torch.empty_like(vp_out)
    lib = m.lib
    P = lambda x: ctypes.c_void_p(x.data_ptr()) if x is not None else None
    Jc = ctypes.c_double()

    def step(wav_d, obs_d):
        """One inversion iteration through the C ABI."""
        m._rc(lib.bh_forward(m.h, P(wav_d), P(seis)))
        m._rc(lib.bh_residual_misfit(m.h, P(seis), P(obs_d), P(resid), ctypes.byref(Jc)))
        m._rc(lib.bh_adjoint_gradient(m.h, P(resid), P(g[0]), P(g[1]), P(g_rho)))
        m._rc(lib.bh_precondition(m.h, P(g[0]), P(g[1]), ctypes.c_double(1e-3)))
        m._rc(lib.bh_update(m.h, P(g[0]), P(g[1]), ctypes.c_double(0.02), None, P(vp_out),
                            P(vs_out)))
        return Jc.value

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- device-resident inputs
    for _ in range(warmup):
        step(wav, obs)
    m.set_model(*start_model)
    torch.cuda.synchronize()
    m.profile(PROFILE_EVERY)
    m.profile_reset()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = m.info("kernel_launches")
    Js = []
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(steps):
            Js.append(step(wav, obs))
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    launches = int(m.info("kernel_launches") - launches0)  # this library's kernels, timed steps
    prof = m.profile_read()
    m.profile(0)

    # ---- end to end: host inputs copied in, result copied out, every step
    wav_h = torch.from_numpy(w.wavelet).pin_memory()
    obs_h = obs.cpu().pin_memory()
    vp_h = torch.empty(shape, dtype=torch.float32).pin_memory()
    vs_h = torch.empty_like(vp_h)
    wav_d = torch.empty_like(wav)
    obs_d = torch.empty_like(obs)
    m.set_model(*start_model)
    torch.cuda.synchronize()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(e2e_steps):
        wav_d.copy_(wav_h, non_blocking=True)
        obs_d.copy_(obs_h, non_blocking=True)
        step(wav_d, obs_d)
        vp_h.copy_(vp_out, non_blocking=True)
        vs_h.copy_(vs_out, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = max_over_ranks(f0.elapsed_time(f1), world, dev)
    h2d = wav_h.numel() * 4 + obs_h.numel() * 4
    d2h = 8 + vp_h.numel() * 4 * 2

    cells_per_step = 2.0 * w.cell_steps()          # forward + adjoint cell updates (useful work)
    value = job_rate(cells_per_step * steps, world, ms)
    grads_per_s = world * w.nshots * steps / (ms / 1e3)
    value_e2e = job_rate(cells_per_step * e2e_steps, world, ms_e2e)

    # ---- roofline of the dominant kernel (largest sampled time)
    peak, peak_kind = measured_peaks()
    s = shot_pml_fraction(w)
    shared = w.nshots > 1
    prof = {k: v for k, v in prof.items() if v[1]}
    dom = max(prof, key=lambda k: prof[k][0])
    win_cells = sum(w.nr * sh["nz"] for sh in w.shots)   # one pass over every window
    recompute = m.info("recompute_steps")
    L = m.info("history_steps")
    fwd_steps = w.nt + recompute
    # forward steps that store history: every step when all are stored,
    # else each segment once when it is re-run before its adjoint
    hist_frac = 1.0 if L >= w.nt else w.nt / fwd_steps
    ngroups = (w.nshots + 31) // 32

    def kernel_cells(k):
        """cells the sampled launches of kernel k processed in the timed region"""
        if k == "fwd_persist":
            return win_cells * fwd_steps * steps
        if k == "adj_persist":
            return win_cells * w.nt * steps
        # one launch per half-step and shot group: the sampled steps launch
        # every group once, and the groups together cover every window
        return win_cells * prof[k][1] / ngroups

    def per_cell(k, model):
        hf = hist_frac if k.startswith("fwd") else 1.0
        if model == "method":
            return sum(method_bytes_per_cell(p, s, shared, hf) for p in PERSIST_PARTS[k])
        if k == "fwd_step":
            return all_array_bytes_per_cell(k, s, with_rho, hf)
        return sum(all_array_bytes_per_cell(p, s, with_rho, hf) for p in PERSIST_PARTS[k])

    kernels = {}
    for k, (tms, nl) in prof.items():
        cells = kernel_cells(k)
        sec = tms / 1e3
        kernels[k] = {"avg_us": 1e3 * tms / nl, "sampled_launches": nl,
                      "cells_per_launch": cells / nl,
                      "alg_bytes_per_launch": per_cell(k, "method") * cells / nl,
                      "alg_GBps": per_cell(k, "method") * cells / sec / 1e9,
                      "all_array_GBps": per_cell(k, "all") * cells / sec / 1e9}
    achieved = kernels[dom]["alg_GBps"]
    dram_per_cell = ncu_traffic(dom, w.name)
    ws = state_bytes_per_group(w)
    if ws > L2_BYTES:
        bound = "hbm"
        bound_note = (f"window state of one shot group {ws / 1e9:.2f} GB > L2 129 MB: "
                      "the state streams from HBM every half-step")
    else:
        bound = "l2"
        bound_note = (f"window state {ws / 1e6:.0f} MB < L2 129 MB: the state stays in L2 "
                      "and DRAM carries the forward history; latency- and barrier-bound, "
                      "the HBM fraction is algorithmic bytes over time")
    roofline = {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak if achieved else None,
                "traffic": (dram_per_cell * kernels[dom]["cells_per_launch"]
                            if dram_per_cell is not None else None),
                "alg_bytes_per_cell_step": per_cell(dom, "method"),
                "frac_all_arrays": kernels[dom]["all_array_GBps"] / peak,
                "all_array_bytes_per_cell_step": per_cell(dom, "all"),
                "peak_source": f"{peak_kind} (hbm_gbs)", "note": bound_note}
    step_bytes = (sum(method_bytes_per_cell(k, s, shared, hist_frac)
                      for k in PERSIST_PARTS["fwd_persist"]) * win_cells * fwd_steps +
                  sum(method_bytes_per_cell(k, s, shared)
                      for k in PERSIST_PARTS["adj_persist"]) * win_cells * w.nt)
    out = {"value": value, "ms_per_step": ms / steps, "config": workload_config(w),
           "gradient_evals_per_s": grads_per_s,
           "step_alg_GBps": world * step_bytes * steps / (ms / 1e3) / 1e9,
           "step_frac": world * step_bytes * steps / (ms / 1e3) / 1e9 / peak,
           "roofline": roofline, "kernels": kernels,
           "e2e": {"value": value_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e / e2e_steps,
                   "steps": e2e_steps},
           "gpu_launches": launches,
           "clocks": clk.summary(), "J_first_last": [Js[0], Js[-1]],
           "history": {k: m.info(k) for k in ("history_steps", "snapshots", "recompute_steps",
                                              "snapshot_precision", "history_snapshot_bytes",
                                              "tiles", "persistent_blocks_fwd",
                                              "persistent_blocks_adj")},
           "gradients": "lambda, mu and rho" if with_rho else "lambda and mu (rho known)",
           "launch": {"group": m.info("group"), "persistent": m.info("persistent"),
                      "tile_code": m.info("tile_code"), "tuning": tuning}}
    m.close()
    return out


def snapshot_study(w, dev, cap):
    """One gradient of the start model per checkpoint-snapshot precision
    (FP32, BF16, FP16) under the same byte cap: relative L2 of the BF16 and
    FP16 gradients and misfits against the FP32-snapshot run (which equals
    the store-every-step result bit for bit)."""
    import numpy as np
    import torch

    from paper_2005_00281_gb300.bh import model_from_workload

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    true = model_from_workload(w, device=dev, checkpoint_cap_bytes=cap)
    true.set_model(t(w.vp_true), t(w.vs_true), t(w.rho_true))
    wav = t(w.wavelet)
    obs = true.forward(wav).clone()
    true.close()
    out, ref = {}, None
    for name, prec in (("fp32", 0), ("bf16", 1), ("fp16", 2)):
        m = model_from_workload(w, device=dev, checkpoint_cap_bytes=cap, snapshot_precision=prec)
        m.tune(steps=32)
        t0 = time.perf_counter()
        seis = m.forward(wav)
        resid, J = m.residual_misfit(seis, obs)
        g = m.adjoint_gradient(resid, with_rho=False)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        gl, gm = g[0].cpu().numpy(), g[1].cpu().numpy()
        row = {"J": J, "seconds": sec, "snapshots": m.info("snapshots"),
               "history_steps": m.info("history_steps"), "tail_steps": m.info("tail_steps"),
               "recompute_steps": m.info("recompute_steps")}
        if ref is None:
            ref = (gl, gm, J)
        else:
            rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
            row["g_lam_rel_l2_vs_fp32"] = rel(gl, ref[0])
            row["g_mu_rel_l2_vs_fp32"] = rel(gm, ref[1])
            row["J_rel_vs_fp32"] = abs(J - ref[2]) / abs(ref[2])
        out[name] = row
        m.close()
    return out


def run_gpu(args, w):
    import torch
    import torch.distributed as dist

    from paper_2005_00281_gb300.build import build_library

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    build_library()

    if world > 1 and rank > 0:
        # every rank inverts its own independent workload: same sizes, other seed
        w = apply_overrides(rank_workload(args.config, rank), args)

    cap_gb = DEFAULT_CAP_GB[args.config] if args.cap_gb is None else args.cap_gb
    snap = args.snap or DEFAULT_SNAP.get(args.config, "fp32")
    prec = {"fp32": 0, "bf16": 1, "fp16": 2}[snap]
    res = measure(w, args, dev, world, rank, args.steps, args.warmup, int(cap_gb * 1e9), prec,
                  args.with_rho, min(args.steps, E2E_STEPS), w.name)
    line = {"metric": METRIC, "value": res.pop("value"), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": res.pop("config")}
    line["config"]["checkpoint_cap_gb"] = cap_gb
    line["config"]["snapshots"] = snap
    line.update(res)
    line["source_sha"] = source_sha()
    if args.compare_snapshots:
        line["snapshot_precision_study"] = snapshot_study(w, dev, int(cap_gb * 1e9))
    if args.secondary and args.config != "c1" and not args.nt and not args.shots:
        from synthetic import PRESETS
        w1 = PRESETS["c1"](seed=rank)
        sec = measure(w1, args, dev, world, rank, min(args.steps, SECONDARY_STEPS),
                      min(args.warmup, 3), 0, 0, args.with_rho, 1, "c1")
        line["secondary_c1"] = {
            "value": sec["value"], "unit": UNIT, "ms_per_step": sec["ms_per_step"],
            "steps": min(args.steps, SECONDARY_STEPS), "config": sec["config"],
            "gradient_evals_per_s": sec["gradient_evals_per_s"], "roofline": sec["roofline"],
            "kernels": sec["kernels"], "step_frac": sec["step_frac"], "clocks": sec["clocks"],
            "gpu_launches": sec["gpu_launches"]}
    if rank == 0 and not args.no_cpu_baseline:
        v, sec_s, threads = oracle_sample(w, CPU_SAMPLE_STEPS)
        line["cpu_baseline"] = {
            "value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first shot of {w.name}, nt truncated to {CPU_SAMPLE_STEPS} of {w.nt} "
                      f"steps (forward + adjoint + gradient, {sec_s:.1f} s); forward loops "
                      f"OpenMP on {threads} threads, adjoint serial"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def apply_overrides(w, args):
    """--nt and --shots applied to a workload (every rank applies the same)."""
    from synthetic import ricker
    if args.nt:
        w.nt = args.nt
        w.wavelet = ricker(w.nt, w.dt, w.f0)
    if args.shots:
        w.shots = w.shots[args.first_shot: args.first_shot + args.shots]
    return w


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--config", default="c2",
                    choices=["c0", "c1", "c2", "c3", "c4", "flushed", "tool"])
    ap.add_argument("--cap-gb", type=float, default=None,
                    help="checkpoint cap in GB (0: store every step of the forward history; "
                         "default per workload: c2 240, c3 4, c4 60, else 0)")
    ap.add_argument("--snap", default=None, choices=["fp32", "bf16", "fp16"],
                    help="precision of the checkpoint snapshots (default fp32; c4 bf16)")
    ap.add_argument("--with-rho", action="store_true",
                    help="also compute the density gradient (the iteration does not use it)")
    ap.add_argument("--no-secondary", dest="secondary", action="store_false",
                    help="skip the secondary single-shot (c1) line")
    ap.add_argument("--compare-snapshots", action="store_true",
                    help="also compute one gradient per snapshot precision and report the "
                         "BF16 / FP16 errors against the FP32-snapshot gradient")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch configuration (no autotuner)")
    ap.add_argument("--opt", action="append",
                    help="library option key=value set after the autotuner (repeatable)")
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner cache file (default: the one in the package)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--per-step", action="store_true",
                    help="one kernel launch per half-step for every run")
    ap.add_argument("--persistent", action="store_true",
                    help="one cooperative launch per run for every shot group (default: "
                         "only where a group's tiles fit the co-resident blocks)")
    ap.add_argument("--nt", type=int, default=None,
                    help="override the step count (small cases for ncu captures only)")
    ap.add_argument("--shots", type=int, default=None,
                    help="keep K shots of a batched workload (a sub-batch), from --first-shot")
    ap.add_argument("--first-shot", type=int, default=0,
                    help="index of the first shot kept by --shots")
    return ap.parse_args(argv)


def main():
    args = parse_args()
    from synthetic import PRESETS
    w = PRESETS[args.config](seed=0)
    apply_overrides(w, args)
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
