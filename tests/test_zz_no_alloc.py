"""bh_residual_misfit_noalloc against bh_residual_misfit, through the C ABI.

The allocation-free entry point serves callers that may not allocate device
memory (another allocator owns the device memory, or allocation is forbidden
after warm-up because it can synchronise the device).  It must give what the model-based entry
point gives on the same inputs: the same residual (one FP32 subtraction per
sample, so bit-identical) and the same FP64 misfit up to summation order.
Two calls in a row check that the shared scratch left by the first call does
not leak into the second.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from synthetic import tiny_borehole

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_00281_gb300 import bh
    bh.load_library()
    return torch, bh


def _noalloc(bh, torch, mod, obs, resid):
    """Direct C-ABI call with caller-owned buffers only."""
    lib = bh.load_library()
    J = ctypes.c_double()
    rc = lib.bh_residual_misfit_noalloc(
        ctypes.c_void_p(mod.data_ptr()), ctypes.c_void_p(obs.data_ptr()),
        ctypes.c_void_p(resid.data_ptr()), mod.numel(), ctypes.byref(J),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.bh_last_error(None)
    return J.value


def test_noalloc_matches_model_entry_point(env):
    torch, bh = env
    # 13 receivers x 6000 steps = 78000 samples: 20 blocks of the reduction
    w = tiny_borehole(seed=7, nt=6000, nrec=13, nz=64)
    m = bh.model_from_workload(w)
    rng = np.random.default_rng(11)
    shape = m.seis_shape()
    for call in range(2):
        mod = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
        obs = torch.from_numpy((rng.standard_normal(shape) * (1 + call)).astype(np.float32)).cuda()
        ref_resid, ref_J = m.residual_misfit(mod, obs)
        resid = torch.full_like(mod, float("nan"))
        J = _noalloc(bh, torch, mod, obs, resid)
        torch.cuda.synchronize()
        assert torch.equal(resid, ref_resid), call
        assert J == pytest.approx(ref_J, rel=1e-12), (call, J, ref_J)
        # the residual may overwrite the modelled data in place
        inplace = mod.clone()
        J2 = _noalloc(bh, torch, inplace, obs, inplace)
        torch.cuda.synchronize()
        assert torch.equal(inplace, ref_resid) and J2 == J, call
    m.close()


def test_noalloc_rejects_oversize(env):
    torch, bh = env
    lib = bh.load_library()
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    J = ctypes.c_double()
    # the size check comes before any device access
    rc = lib.bh_residual_misfit_noalloc(
        ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
        ctypes.c_void_p(x.data_ptr()), bh.NOALLOC_MAX_SAMPLES + 1, ctypes.byref(J),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1
    assert b"exceed" in lib.bh_last_error(None)
