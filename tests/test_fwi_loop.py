"""Host logic of the inversion loop (paper_2005_00281_gb300.fwi.run): the stop
rule of the Method section and the backtracking safeguard, on a stand-in
model whose misfit is a weighted quadratic (no GPU: every call the loop makes
is answered on the host)."""
import numpy as np
import pytest
import torch

from paper_2005_00281_gb300 import fwi


class QuadModel:
    """seis = x, J = 1/2 sum w (x - x_obs)^2; the step is kappa max|x| / max|g|
    along the gradient, like the library's update (Eq. 11, Eq. 12)."""

    def __init__(self, x0, w):
        self.x = x0.clone()
        self.w = w
        self.forwards = 0

    def empty_seis(self):
        return torch.empty_like(self.x)

    def forward(self, wavelet, seis):
        self.forwards += 1
        seis.copy_(self.x)
        return seis

    def residual_misfit(self, seis, obs, resid):
        resid.copy_(seis - obs)
        return resid, float(0.5 * (self.w * resid * resid).sum())

    def adjoint_gradient(self, resid, with_rho=True):
        g = (self.w * resid).double()
        return g, g.clone(), (g.clone() if with_rho else None)

    def precondition(self, g_lam, g_mu, eps_rel=1e-3):
        return g_lam, g_mu

    def update(self, g_lam, g_mu, kappa=0.02, want_velocities=True):
        a = kappa * float(self.x.abs().max()) / float(g_lam.abs().max())
        self.x -= (a * g_lam).float()
        return (a, a), None, None

    def update_velocity(self, g_lam, g_mu, g_rho=None, update_rho=False, kappa=0.02,
                        want_model=True):
        (a, _), _, _ = self.update(g_lam, g_mu, kappa)
        return (a, a, 0.0), None, None, None

    def velocities(self):
        return self.x.clone(), self.x.clone()

    def density(self):
        return torch.ones_like(self.x)

    def set_model(self, vp, vs, rho):
        self.x.copy_(vp)


def _problem():
    rng = np.random.default_rng(3)
    obs = torch.from_numpy(rng.uniform(2.0, 3.0, 64).astype(np.float32))
    x0 = obs * torch.from_numpy(rng.uniform(0.8, 1.2, 64).astype(np.float32))
    w = torch.from_numpy(rng.uniform(0.1, 1.0, 64).astype(np.float32))
    w[7] = 40.0   # one stiff direction: a large fixed step overshoots along it
    return x0, w, obs


@pytest.mark.parametrize("param", ["lame", "velocity"])
def test_backtracking_keeps_the_misfit_falling(param):
    x0, w, obs = _problem()
    plain = QuadModel(x0, w)
    st0 = fwi.run(plain, None, obs, 12, kappa=0.5, param=param)
    assert any(b > a for a, b in zip(st0.J, st0.J[1:])), "the fixed step should overshoot here"
    m = QuadModel(x0, w)
    st = fwi.run(m, None, obs, 40, kappa=0.5, param=param, backtrack=True)
    assert st.rejected > 0 and st.kappa == 0.5 * 0.5 ** st.rejected
    assert all(b < a for a, b in zip(st.J, st.J[1:]))
    assert m.forwards == 40 and st.iteration == 40 - st.rejected
    assert len(st.alpha) == st.iteration == len(st.seconds)
    assert st.J[-1] < 0.05 * st.J[0]


def test_stop_rule_relative_threshold():
    x0, w, obs = _problem()
    w[7] = 1.0
    m = QuadModel(x0, w)
    st = fwi.run(m, None, obs, 200, kappa=0.05, rel_threshold=0.1)
    # stops at the first misfit at or below a tenth of the first one; that
    # misfit is recorded, no step follows it
    assert st.J[-1] <= 0.1 * st.J[0] and all(j > 0.1 * st.J[0] for j in st.J[:-1])
    assert st.iteration == len(st.J) - 1 and m.forwards == len(st.J)


def test_state_resumes(tmp_path):
    x0, w, obs = _problem()
    m = QuadModel(x0, w)
    st = fwi.run(m, None, obs, 6, kappa=0.5, backtrack=True)
    path = str(tmp_path / "s.npz")
    fwi.save(path, m, st, m.density())
    m2 = QuadModel(torch.zeros_like(x0), w)
    st2, _ = fwi.load(path, m2, device="cpu")
    assert st2.iteration == st.iteration and st2.rejected == st.rejected
    assert st2.kappa == st.kappa and np.allclose(st2.J, st.J)
    assert torch.equal(m2.x, m.x)
