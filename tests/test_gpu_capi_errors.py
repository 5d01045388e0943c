"""Error paths of the C ABI: status codes, no aborts."""
import numpy as np
import pytest

from synthetic import tiny_borehole

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bhmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_00281_gb300 import bh
    bh.load_library()
    return bh


def _args(w):
    import torch
    t = lambda a: torch.from_numpy(a).cuda()
    return (w.nr, w.nz, w.nt, w.npml_r, w.npml_z, w.dr, w.dz, w.dt, w.f0, t(w.vp), t(w.vs),
            t(w.rho), w.shots)


def test_cfl_violation(bhmod):
    w = tiny_borehole(seed=0, nt=10)
    a = list(_args(w))
    a[7] = 5e-6  # dt far above the stability limit
    with pytest.raises(bhmod.BhError) as e:
        bhmod.Model(*a)
    assert e.value.status == 2


def test_receiver_outside_window(bhmod):
    w = tiny_borehole(seed=0, nt=10)
    w.shots[0]["rec_iz"] = [w.nz - 1]
    with pytest.raises(bhmod.BhError) as e:
        bhmod.Model(*_args(w))
    assert e.value.status == 1


def test_window_outside_model(bhmod):
    w = tiny_borehole(seed=0, nt=10)
    w.shots[0]["z_offset"] = 5
    with pytest.raises(bhmod.BhError) as e:
        bhmod.Model(*_args(w))
    assert e.value.status == 1


def test_call_order(bhmod):
    import torch
    w = tiny_borehole(seed=0, nt=10)
    m = bhmod.Model(*_args(w))
    resid = torch.zeros(m.seis_shape(), dtype=torch.float32, device="cuda")
    with pytest.raises(bhmod.BhError) as e:
        m.adjoint_gradient(resid)
    assert e.value.status == 6
    g = torch.zeros((w.nr, w.nz), dtype=torch.float64, device="cuda")
    with pytest.raises(bhmod.BhError) as e:
        m.precondition(g, g.clone())
    assert e.value.status == 6
    m.close()


def test_unsupported_options(bhmod):
    w = tiny_borehole(seed=0, nt=10)
    with pytest.raises(bhmod.BhError) as e:
        bhmod.Model(*_args(w), snapshot_precision=3)
    assert e.value.status in (1, 7)
