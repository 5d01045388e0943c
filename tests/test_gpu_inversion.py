"""The paper's inversion experiments on stand-in models (Numerical
Examples): the diagonal preconditioner's suppression of the near-wall
gradient (Fig. 6), and an inversion of a flushed-zone model (Fig. 7) from a
start model built from the wall and far velocity logs (Fig. 3, Fig. 4), run
to a misfit threshold."""
import numpy as np
import pytest

from synthetic import config0
from synthetic.workloads import flushed_zone
from tests.gpu_common import gpu_gradient

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_00281_gb300.bh import load_library
    load_library()
    return torch


def _band(w, a, r0, r1):
    r = (np.arange(w.nr) + 0.5) * w.dr
    rows = (r >= r0) & (r < r1)
    cols = slice(w.npml_z, w.nz - w.npml_z)
    return float(np.mean(np.abs(a[rows, cols])))


def test_preconditioner_suppresses_the_near_wall_gradient(cuda):
    """Fig. 6: guided waves along the fluid-solid wall make the raw lambda
    gradient large next to the wall; the pseudo-Hessian is large there too,
    so after preconditioning the near-wall band (0.10-0.15 m) weighs less
    against the band 0.30-0.50 m than before."""
    torch = cuda
    from tests.gpu_common import oracle_observed
    w = config0()
    obs = oracle_observed(w)
    m, gpu = gpu_gradient(w, obs)
    g_raw = gpu["g_lam"]
    gl = torch.from_numpy(g_raw.copy()).cuda()
    gm = torch.from_numpy(gpu["g_mu"].copy()).cuda()
    m.precondition(gl, gm, 1e-3)
    g_pre = gl.cpu().numpy()
    H = gpu["H_lam"]
    m.close()
    raw = _band(w, g_raw, 0.10, 0.15) / _band(w, g_raw, 0.30, 0.50)
    pre = _band(w, g_pre, 0.10, 0.15) / _band(w, g_pre, 0.30, 0.50)
    hr = _band(w, H, 0.10, 0.15) / _band(w, H, 0.30, 0.50)
    print(f"near/far band ratio of |g_lambda|: raw {raw:.3g}, preconditioned {pre:.3g}; "
          f"pseudo-Hessian {hr:.3g}")
    assert raw > 1.0 and hr > 1.0
    assert pre < 0.5 * raw


def test_flushed_zone_inversion_to_threshold(cuda):
    """A reduced flushed-zone model (two shots, 3000 steps): start model from
    the wall and one-meter velocity logs (bh_starting_model), preconditioned
    velocity-space steps until the misfit halves (the stop rule) or 8
    iterations: J falls every iteration and reaches the threshold.  The
    model error over the formation is printed (a few small steps do not
    lower it everywhere: most cells are far from the wave paths)."""
    torch = cuda
    from paper_2005_00281_gb300 import fwi
    from paper_2005_00281_gb300.bh import model_from_workload, starting_model

    w = flushed_zone(seed=1, nshots=2, nt=3000, nz_window=1400)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    lg = w.logs
    vp0, vs0 = starting_model(w.nr, w.dr, lg["r_wall"], lg["r_far"], t(lg["vp_wall"]),
                              t(lg["vs_wall"]), t(lg["vp_far"]), t(lg["vs_far"]))
    truth = model_from_workload(w)
    truth.set_model(t(w.vp_true), t(w.vs_true), t(w.rho_true))
    wav = t(w.wavelet)
    obs = truth.forward(wav).clone()
    truth.close()
    m = model_from_workload(w)
    m.set_model(vp0, vs0, t(w.rho))
    vt = w.vp_true
    formation = (w.vs_true > 0) & (np.arange(w.nr)[:, None] < w.nr - w.npml_r)
    formation[:, :w.npml_z] = False
    formation[:, w.nz - w.npml_z:] = False
    err = lambda v: float(np.linalg.norm((v - vt)[formation]) / np.linalg.norm(vt[formation]))
    e0 = err(vp0.cpu().numpy())
    st = fwi.run(m, wav, obs, 8, kappa=0.01, rel_threshold=0.5, param="velocity")
    vp1, _ = m.velocities()
    e1 = err(vp1.cpu().numpy())
    m.close()
    print(f"flushed zone: J {st.J[0]:.4g} -> {st.J[-1]:.4g} in {st.iteration} iterations; "
          f"Vp rel. error {e0:.4g} -> {e1:.4g}")
    assert all(b < a for a, b in zip(st.J, st.J[1:]))
    assert st.J[-1] <= 0.5 * st.J[0] and st.iteration < 8
