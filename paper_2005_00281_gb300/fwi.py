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
    kappa: float = 0.0     # step factor in force (backtracking halves it); 0: not yet set
    rejected: int = 0      # trial steps that raised the misfit (backtracking)


def save(path, model, state: FwiState, rho):
    vp, vs = model.velocities()
    np.savez(path, vp=vp.cpu().numpy(), vs=vs.cpu().numpy(), rho=rho.cpu().numpy(),
             iteration=state.iteration, J=np.array(state.J), alpha=np.array(state.alpha),
             seconds=np.array(state.seconds), kappa=state.kappa, rejected=state.rejected)


def load(path, model, device="cuda"):
    d = np.load(path)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
    rho = t(d["rho"])
    model.set_model(t(d["vp"]), t(d["vs"]), rho)
    st = FwiState(int(d["iteration"]), list(d["J"]), [tuple(a) for a in d["alpha"]],
                  list(d["seconds"]), float(d["kappa"]) if "kappa" in d else 0.0,
                  int(d["rejected"]) if "rejected" in d else 0)
    return st, rho


def _step(model, g, param, update_rho, kappa):
    """One model update along the (preconditioned) gradient g."""
    if param == "velocity":
        alpha, _, _, _ = model.update_velocity(g[0], g[1], g[2], update_rho=update_rho,
                                               kappa=kappa, want_model=False)
    else:
        alpha, _, _ = model.update(g[0], g[1], kappa, want_velocities=False)
    return alpha


def run(model, wavelet, seis_obs, iterations, *, kappa=0.02, eps_rel=1e-3, threshold=0.0,
        rel_threshold=0.0, precondition=True, param="lame", update_rho=False,
        backtrack=False, state: FwiState | None = None, checkpoint_path=None, rho=None,
        log=None):
    """Run up to `iterations` more forward modellings, each followed by an
    inversion step, stopping once the misfit falls to `threshold` or to
    `rel_threshold` times the first iteration's (the stop rule of the Method
    section).  param "lame" steps lambda and mu (Eq. 9, Eq. 10); "velocity"
    steps Vp, Vs and, with update_rho, rho; the step is kappa times the
    largest model value over the largest gradient (Eq. 11, Eq. 12).

    backtrack: a safeguard the paper does not state.  A step after which the
    misfit is higher than before is taken back: the model returns to the last
    accepted one, kappa is halved and the step is retried along the same
    gradient (one forward modelling per retry, no new gradient).  Without it
    every step is kept, as in the plain method.  Returns the FwiState."""
    st = state or FwiState()
    if st.kappa <= 0.0:
        st.kappa = kappa
    seis = model.empty_seis()
    resid = torch.empty_like(seis)
    want_rho = param == "velocity" and update_rho
    last = None  # (model, preconditioned gradient) of the last accepted iteration
    for _ in range(iterations):
        t0 = time.perf_counter()
        model.forward(wavelet, seis)
        _, J = model.residual_misfit(seis, seis_obs, resid)
        if backtrack and last is not None and J > st.J[-1]:
            st.rejected += 1
            st.kappa *= 0.5
            model.set_model(*last[0])
            alpha = _step(model, last[1], param, update_rho, st.kappa)
            st.alpha[-1] = alpha
            st.seconds[-1] += time.perf_counter() - t0
            if log:
                log(f"iteration {st.iteration}: trial J = {J:.6e} rejected, kappa -> {st.kappa:.3g}")
            continue
        if J <= threshold or (st.J and rel_threshold > 0 and J <= rel_threshold * st.J[0]):
            st.J.append(J)
            break
        g = model.adjoint_gradient(resid, with_rho=want_rho)
        if precondition:
            model.precondition(g[0], g[1], eps_rel)
        if backtrack:
            vp, vs = model.velocities()
            last = ((vp, vs, model.density()), g)
        alpha = _step(model, g, param, update_rho, st.kappa)
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


def main(argv=None):
    """Inversion of a synthetic workload from the command line: the observed
    data are modelled in the true model, the gradient of the misfit with
    respect to Vp (through BhWave, the library's adjoint) is checked against
    central differences at random formation cells and at the formation cells
    of largest gradient (at random cells far from the wave paths a change of
    J is near the FP32 rounding of the seismograms), then `--iterations`
    preconditioned gradient-descent steps run from the start model.  Prints
    one JSON line."""
    import argparse
    import json
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from synthetic import PRESETS

    from .autograd import BhWave, misfit
    from .bh import model_from_workload

    ap = argparse.ArgumentParser(prog="python -m paper_2005_00281_gb300.fwi")
    ap.add_argument("--config", default="c3", choices=sorted(PRESETS))
    ap.add_argument("--iterations", type=int, default=10)
    ap.add_argument("--cap-gb", type=float, default=4.0, help="checkpoint cap (0: store all)")
    ap.add_argument("--fd-cells", type=int, default=32)
    ap.add_argument("--fd-step", type=float, default=1e-2, help="relative Vp change")
    ap.add_argument("--kappa", type=float, default=0.02)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--start", default="workload", choices=["workload", "logs"],
                    help="start model: the workload's, or the velocity logs at the wall and "
                         "one meter beyond interpolated in r (bh_starting_model)")
    ap.add_argument("--rel-threshold", type=float, default=0.0,
                    help="stop once J falls to this fraction of the first iteration's")
    ap.add_argument("--param", default="lame", choices=["lame", "velocity"])
    ap.add_argument("--no-precondition", dest="precondition", action="store_false")
    ap.add_argument("--backtrack", action="store_true",
                    help="take back a step that raises the misfit and halve kappa")
    ap.add_argument("--near-wall", type=float, default=0.4,
                    help="radial extent (m) beyond the wall of the near-wall model error")
    args = ap.parse_args(argv)
    if not torch.cuda.is_available():
        raise SystemExit("the inversion needs a CUDA device (there is no CPU fallback)")
    w = PRESETS[args.config]() if args.config == "c0" else PRESETS[args.config](seed=args.seed)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    if args.start == "logs":
        from .bh import starting_model
        if w.logs is None:
            raise SystemExit(f"workload {args.config} has no velocity logs")
        lg = w.logs
        vp_s, vs_s = starting_model(w.nr, w.dr, lg["r_wall"], lg["r_far"], t(lg["vp_wall"]),
                                    t(lg["vs_wall"]), t(lg["vp_far"]), t(lg["vs_far"]))
        w.vp, w.vs = vp_s.cpu().numpy(), vs_s.cpu().numpy()
    cap = int(args.cap_gb * 1e9)
    m = model_from_workload(w, checkpoint_cap_bytes=cap)
    wav = t(w.wavelet)
    with torch.no_grad():
        obs = BhWave.apply(t(w.vp_true), t(w.vs_true), t(w.rho_true), m, wav).clone()

    # gradient of J with respect to Vp at the start model, against central differences
    fd_rows, fd_err, rel = [], None, [float("nan")]
    if args.fd_cells > 0:
        fd_rows, fd_err, rel = _fd_check(args, w, m, wav, obs, t)

    # the inversion loop from the start model
    vs, rho = t(w.vs), t(w.rho)
    m.set_model(t(w.vp), vs, rho)
    mask = ((w.vs > 0) & (np.arange(w.nr)[:, None] < w.nr - w.npml_r) &
            (np.arange(w.nz)[None, :] >= w.npml_z) & (np.arange(w.nz)[None, :] < w.nz - w.npml_z))
    # the near-wall zone: formation rows within --near-wall metres of the wall
    i_wall = int(np.argmax(w.vs[:, w.nz // 2] > 0))
    near = mask & (np.arange(w.nr)[:, None] < i_wall + int(round(args.near_wall / w.dr)))

    def model_error():
        vp_c, vs_c = m.velocities()
        vp_c, vs_c = vp_c.cpu().numpy(), vs_c.cpu().numpy()
        e = lambda a, b, k: float(np.linalg.norm((a - b)[k]) / np.linalg.norm(b[k]))
        return {"vp": e(vp_c, w.vp_true, mask), "vs": e(vs_c, w.vs_true, mask),
                "vp_near_wall": e(vp_c, w.vp_true, near), "vs_near_wall": e(vs_c, w.vs_true, near)}

    err0 = model_error()
    st = run(m, wav, obs, args.iterations, kappa=args.kappa, rel_threshold=args.rel_threshold,
             precondition=args.precondition, param=args.param, backtrack=args.backtrack,
             log=lambda s: print(s, file=sys.stderr, flush=True))
    err1 = model_error()
    info = {k: m.info(k) for k in ("history_steps", "snapshots", "tail_steps", "recompute_steps",
                                   "history_snapshot_bytes")}
    m.close()
    print(json.dumps({
        "workload": args.config, "nr": w.nr, "nz": w.nz, "nt": w.nt, "nshots": w.nshots,
        "start": args.start, "param": args.param, "precondition": args.precondition,
        "rel_threshold": args.rel_threshold, "iterations_run": st.iteration,
        "backtrack": args.backtrack, "rejected_steps": st.rejected, "kappa_start": args.kappa,
        "kappa_end": st.kappa, "near_wall_m": args.near_wall,
        "model_rel_error_start": err0, "model_rel_error_end": err1,
        "checkpoint": info, "J": [float(x) for x in st.J],
        "seconds_per_iteration": [float(x) for x in st.seconds],
        "fd_check": {"cells": args.fd_cells, "relative_step": args.fd_step,
                     "max_abs_error_over_max_gradient": fd_err,
                     "largest_cells_relative_error_median": float(np.median(rel)),
                     "largest_cells_relative_error_max": float(np.max(rel)),
                     "rows_random": [list(r) for r in fd_rows[: args.fd_cells]],
                     "rows_largest": [list(r) for r in fd_rows[args.fd_cells:]]}}), flush=True)


def _fd_check(args, w, m, wav, obs, t):
    """Central differences of J in Vp at random formation cells and at the
    cells of largest gradient, against BhWave's gradient."""
    from .autograd import BhWave, misfit
    vp = t(w.vp).requires_grad_(True)
    vs, rho = t(w.vs), t(w.rho)
    J0 = misfit(BhWave.apply(vp, vs, rho, m, wav), obs, m)
    J0.backward()
    g = vp.grad.detach().cpu().numpy()
    rng = np.random.default_rng(args.seed)
    form = np.argwhere((w.vs > 0) & (np.arange(w.nr)[:, None] < w.nr - w.npml_r) &
                       (np.arange(w.nz)[None, :] >= w.npml_z) &
                       (np.arange(w.nz)[None, :] < w.nz - w.npml_z))
    rand = form[rng.choice(len(form), size=args.fd_cells, replace=False)]
    gform = np.abs(g[form[:, 0], form[:, 1]])
    top = form[np.argsort(gform)[-args.fd_cells:]]
    fd_rows = []
    with torch.no_grad():
        for i, j in np.concatenate([rand, top]):
            h = args.fd_step * float(w.vp[i, j])
            vals = []
            for sgn in (1.0, -1.0):
                vp2 = t(w.vp).clone()
                vp2[i, j] += sgn * h
                vals.append(float(misfit(BhWave.apply(vp2, vs, rho, m, wav), obs, m)))
            fd_rows.append((int(i), int(j), (vals[0] - vals[1]) / (2 * h), float(g[i, j])))
    gmax = float(np.abs(g).max())
    fd_err = max(abs(fd - ad) for _, _, fd, ad in fd_rows) / gmax
    rel = [abs(fd - ad) / abs(ad) for _, _, fd, ad in fd_rows[args.fd_cells:]]
    return fd_rows, fd_err, rel


if __name__ == "__main__":
    main()
