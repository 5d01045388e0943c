"""Differentiable wrapper and the inversion loop on the GPU."""
import numpy as np
import pytest

from synthetic import tiny_borehole

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_autograd_matches_finite_differences(torch_cuda):
    """BhWave.backward (discrete adjoint) against central differences of the
    FP32 forward at 32 random formation cells."""
    torch = torch_cuda
    from paper_2005_00281_gb300.autograd import BhWave, misfit
    from paper_2005_00281_gb300.bh import model_from_workload

    w = tiny_borehole(seed=12, nt=260)
    m = model_from_workload(w)
    t = lambda a: torch.from_numpy(a).cuda()
    wav = t(w.wavelet)
    with torch.no_grad():
        obs = BhWave.apply(t(w.vp_true), t(w.vs_true), t(w.rho_true), m, wav).clone()
    vp = t(w.vp).requires_grad_(True)
    vs = t(w.vs).requires_grad_(True)
    rho = t(w.rho).requires_grad_(True)
    J = misfit(BhWave.apply(vp, vs, rho, m, wav), obs, m)
    J.backward()
    rng = np.random.default_rng(3)
    cells = [(int(rng.integers(w.nr - w.npml_r - 14, w.nr - w.npml_r)),
              int(rng.integers(w.npml_z, w.nz - w.npml_z))) for _ in range(32)]
    for k, (x, g) in enumerate(((vp, vp.grad), (vs, vs.grad), (rho, rho.grad))):
        scale = float(g.abs().max())
        for (i, j) in cells:
            h = 1e-3 * float(x[i, j])
            vals = []
            for sgn in (1, -1):
                with torch.no_grad():
                    args = [a.detach().clone() for a in (vp, vs, rho)]
                    args[k][i, j] += sgn * h
                    vals.append(float(misfit(BhWave.apply(*args, m, wav), obs, m)))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - float(g[i, j])) <= 2e-2 * scale, (i, j, fd, float(g[i, j]))
    m.close()


def test_fwi_loop_reduces_misfit_and_resumes(torch_cuda, tmp_path):
    torch = torch_cuda
    from paper_2005_00281_gb300 import fwi
    from paper_2005_00281_gb300.bh import model_from_workload

    w = tiny_borehole(seed=13, nt=260)
    t = lambda a: torch.from_numpy(a).cuda()
    truth = model_from_workload(w)
    truth.set_model(t(w.vp_true), t(w.vs_true), t(w.rho_true))
    wav = t(w.wavelet)
    obs = truth.forward(wav).clone()
    truth.close()
    m = model_from_workload(w)
    rho = t(w.rho)
    ck = str(tmp_path / "fwi.npz")
    st = fwi.run(m, wav, obs, 3, kappa=0.01, checkpoint_path=ck, rho=rho)
    assert len(st.J) == 3 and st.J[-1] < st.J[0]
    # resume into a fresh model from the saved state and continue
    m2 = model_from_workload(w)
    st2, rho2 = fwi.load(ck, m2)
    assert st2.iteration == 3
    st2 = fwi.run(m2, wav, obs, 2, kappa=0.01, state=st2)
    assert st2.iteration == 5 and st2.J[-1] < st.J[0]
    m.close()
    m2.close()


def test_backward_checks_the_stored_forward(torch_cuda):
    """The model keeps one forward history: a backward after another forward
    on the same model raises instead of returning the other run's gradient."""
    torch = torch_cuda
    from paper_2005_00281_gb300.autograd import BhWave, misfit
    from paper_2005_00281_gb300.bh import model_from_workload

    w = tiny_borehole(seed=12, nt=120)
    m = model_from_workload(w)
    t = lambda a: torch.from_numpy(a).cuda()
    wav = t(w.wavelet)
    vp = t(w.vp).requires_grad_(True)
    seis = BhWave.apply(vp, t(w.vs), t(w.rho), m, wav)
    J = misfit(seis, torch.zeros_like(seis), m)
    with torch.no_grad():
        BhWave.apply(t(w.vp_true), t(w.vs_true), t(w.rho_true), m, wav)
    with pytest.raises(RuntimeError, match="another forward"):
        J.backward()
    m.close()


def test_misfit_is_the_library_misfit(torch_cuda):
    """BhMisfit's value is bh_residual_misfit's FP64 J and its gradient the
    library's residual."""
    torch = torch_cuda
    from paper_2005_00281_gb300.autograd import misfit
    from paper_2005_00281_gb300.bh import model_from_workload

    w = tiny_borehole(seed=2, nt=64)
    m = model_from_workload(w)
    rng = np.random.default_rng(0)
    shape = m.seis_shape()
    a = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda().requires_grad_(True)
    b = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
    J = misfit(a, b, m)
    resid, J_lib = m.residual_misfit(a.detach(), b)
    assert float(J) == J_lib
    (3.0 * J).backward()
    assert torch.equal(a.grad, 3.0 * resid)
    m.close()
