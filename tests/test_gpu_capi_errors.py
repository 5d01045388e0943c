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


def test_barrier_timeout_is_reported(bhmod):
    """A grid barrier whose wait runs out (it waits for one arrival that
    never comes) makes every block return; the call reports BH_ERR_TIMEOUT
    and the context stays usable."""
    import torch
    w = tiny_borehole(seed=0, nt=20)
    m = bhmod.Model(*_args(w))
    if m.lib.bh_set_option(m.h, b"persistent", 1.0) != 0:
        pytest.skip("no cooperative launch")
    m.set_option("barrier_timeout_ms", 50)
    m.set_option("barrier_extra_arrivals", 1)
    wav = torch.from_numpy(w.wavelet).cuda()
    with pytest.raises(bhmod.BhError) as e:
        m.forward(wav)
    assert e.value.status == 5
    m.set_option("barrier_extra_arrivals", 0)
    seis = m.forward(wav)
    torch.cuda.synchronize()
    assert torch.isfinite(seis).all()
    m.close()


def test_bad_option(bhmod):
    w = tiny_borehole(seed=0, nt=10)
    m = bhmod.Model(*_args(w))
    with pytest.raises(bhmod.BhError) as e:
        m.set_option("no_such_option", 1)
    assert e.value.status == 1
    with pytest.raises(bhmod.BhError) as e:
        m.set_option("persistent", 3)
    assert e.value.status == 1
    m.close()
