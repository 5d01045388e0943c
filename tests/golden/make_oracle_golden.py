"""Writes oracle_tiny.txt: the FP64 oracle's seismograms, misfit and
gradients on a small seeded borehole (24 x 48 cells, 300 steps), so that a
later change of the oracle's arithmetic shows up as a failing test.  Only
the oracle and the seeded input generators run here.

    python tests/golden/make_oracle_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from synthetic import tiny_borehole  # noqa: E402

NT = 300
CELLS = [(0, 20), (3, 12), (4, 20), (5, 25), (10, 15), (12, 24), (16, 30), (9, 40)]


def compute():
    """(J, seis samples, gradient samples) of the golden case, from the oracle."""
    w = tiny_borehole(seed=0, nt=NT)
    sh = w.shots[0]
    g = O.Grid(w.nr, w.nz, w.nt, w.npml_r, w.npml_z, w.dr, w.dz, w.dt, w.f0, w.pml_R)
    obs, _ = O.forward(g, w.vp_true, w.vs_true, w.rho_true, w.wavelet, sh["src"], sh["rec_iz"],
                       store_v=False)
    res = O.shot_gradient(g, w.vp, w.vs, w.rho, w.wavelet, w.shots, obs[None])
    seis = res["seis"][0][:, ::8]
    grads = {k: [float(res[k][i, j]) for (i, j) in CELLS] for k in ("g_lam", "g_mu", "g_rho")}
    return float(res["J"]), seis, grads


def main():
    J, seis, grads = compute()
    lines = ["# FP64 oracle on tiny_borehole(seed=0, nt=300): 24 x 48 cells, 6-cell C-PML,",
             "# 1 cm, dt 1 us, Ricker 15 kHz; data from the true model, gradient at the start",
             "# model.  Written by tests/golden/make_oracle_golden.py (oracle only).",
             f"J {J:.17e}"]
    for r, row in enumerate(seis):
        lines.append(f"seis{r} " + " ".join(f"{v:.17e}" for v in row))
    for k, vals in grads.items():
        lines.append(f"{k} " + " ".join(f"{v:.17e}" for v in vals))
    lines.append("cells " + " ".join(f"{i},{j}" for i, j in CELLS))
    with open(os.path.join(HERE, "oracle_tiny.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
