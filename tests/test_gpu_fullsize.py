"""Checks at the benchmark workloads' full spatial sizes, in the launch
configurations bench.py times (the autotuner's cached choices) and in the
cooperative form.

- The production shot (240 x 1600 cells) against the FP64 oracle element by
  element, with the run shortened to 450 steps and the receivers moved to
  0.1-0.4 m from the source so that the waves reach them (the tile table,
  grid and kernels are the same as in the 8000-step run).  The data are
  zero, so the adjoint source is the whole seismogram: with near receivers
  and a short run the damage-zone residual would be a small difference of
  nearly equal traces, whose relative error is the seismogram's relative
  error (1e-5) times their ratio.
- The full 8000-step run: the adjoint gradient against a central difference
  of the forward misfit along a random direction (a property of the exact
  discrete adjoint at any size), and two runs bit for bit.
- The 400 x 4000 shot under a checkpoint byte cap against storing every step
  (bit for bit), shortened to 1000 steps.
- Two windows of the 64-shot logging run in the launch configuration the
  benchmark takes from the autotuner cache, against the oracle, and the
  whole 64-shot run in that configuration: deterministic, and equal to
  rounding with the half-step forward kernels.
- Two shots of the 256-shot run for every snapshot precision against the
  oracle.
"""
import numpy as np
import pytest

from synthetic import PRESETS
from tests.gpu_common import gpu_gradient, oracle_gradient, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_00281_gb300.bh import load_library
    load_library()
    return torch


def _shortened_c1(nt):
    w = PRESETS["c1"](seed=0)
    w.nt = nt
    w.wavelet = np.ascontiguousarray(w.wavelet[:nt])
    src = w.shots[0]["src"][1]
    w.shots[0]["rec_iz"] = [src + 20 * k for k in range(1, 5)]
    return w


def test_c1_window_parity(cuda, orc):
    """The production window against the oracle in the cooperative form (one
    launch per run over its 750 tiles) and in the configuration the
    autotuner cache holds for it (what bench.py's secondary line times)."""
    torch = cuda
    from paper_2005_00281_gb300 import bh
    w = _shortened_c1(450)
    obs = np.zeros((1, len(w.shots[0]["rec_iz"]), w.nt))
    m, coop = gpu_gradient(w, obs)
    # one cooperative launch for the forward run and one for the adjoint
    assert m.info("tiles") == 750 and m.info("persistent_runs_per_step") == 2
    m.close()
    runs = {"cooperative": coop}
    got = bh.tune_lookup(bh.TUNE_CACHE, torch.cuda.get_device_name(0), w.nr, 1600, 1)
    if got is not None:
        G, form, code, split, order = got
        opts = dict(persistent=form, tile_code=code, split=split, tile_order=order)
        mc, runs["cached"] = gpu_gradient(w, obs, options=opts)
        mc.close()
    ref = oracle_gradient(w, obs)
    assert np.abs(ref["seis"][0]).max() > 0
    for name, gpu in runs.items():
        assert rel_l2(gpu["seis"][0], ref["seis"][0]) <= 1e-5, name
        assert abs(gpu["J"] - ref["J"]) <= 1e-5 * ref["J"], name
        for k in ("g_lam", "g_mu", "g_rho", "H_lam", "H_mu"):
            e = rel_l2(gpu[k], ref[k])
            assert e <= 1e-4, (name, k, e)


def _c1_run(torch, m, w, obs, wav):
    seis = m.forward(wav)
    resid, J = m.residual_misfit(seis, obs)
    g = m.adjoint_gradient(resid)
    torch.cuda.synchronize()
    return J, [x.clone() for x in g]


def test_c1_full_run_gradient_and_determinism(cuda):
    """8000 steps on 240 x 1600 cells: <g, dm> against (J(m + h dm) -
    J(m - h dm)) / 2h for a smooth random change of lambda and mu in the
    formation, and a second run identical bit for bit."""
    torch = cuda
    from paper_2005_00281_gb300.bh import model_from_workload

    w = PRESETS["c1"](seed=0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    truth = model_from_workload(w)
    truth.set_model(t(w.vp_true), t(w.vs_true), t(w.rho_true))
    wav = t(w.wavelet)
    obs = truth.forward(wav).clone()
    truth.close()
    m = model_from_workload(w)
    J0, g = _c1_run(torch, m, w, obs, wav)
    assert m.info("tiles") == 750 and m.info("persistent_runs_per_step") == 2
    J0b, g_b = _c1_run(torch, m, w, obs, wav)
    assert J0 == J0b
    for a, b in zip(g, g_b):
        assert torch.equal(a, b)
    # smooth direction in (lambda, mu) on formation cells away from the layers
    rng = np.random.default_rng(7)
    nr, nz = w.nr, w.nz
    ii, jj = np.meshgrid(np.arange(nr), np.arange(nz), indexing="ij")
    dm = np.zeros((nr, nz))
    for _ in range(6):
        ci, cj = rng.uniform(30, nr - w.npml_r - 30), rng.uniform(w.npml_z + 60, nz - w.npml_z - 60)
        dm += rng.normal() * np.exp(-((ii - ci) ** 2 / 200.0 + (jj - cj) ** 2 / 800.0))
    dm[w.vs <= 0] = 0.0
    dm[nr - w.npml_r:, :] = 0.0
    dm[:, : w.npml_z] = 0.0
    dm[:, nz - w.npml_z:] = 0.0
    lam = w.rho * (w.vp ** 2 - 2 * w.vs ** 2)
    mu = w.rho * w.vs ** 2
    dlam, dmu = 0.5 * lam * dm, 0.5 * mu * dm
    pred = float((g[0].cpu().numpy() * dlam).sum() + (g[1].cpu().numpy() * dmu).sum())
    vals = []
    h = 1e-3
    for sgn in (1, -1):
        lam2, mu2 = lam + sgn * h * dlam, mu + sgn * h * dmu
        vs2 = np.sqrt(np.maximum(mu2, 0) / w.rho)
        vp2 = np.sqrt((lam2 + 2 * mu2) / w.rho)
        m.set_model(t(vp2.astype(np.float32)), t(vs2.astype(np.float32)), t(w.rho))
        seis = m.forward(wav)
        _, J = m.residual_misfit(seis, obs)
        vals.append(J)
    fd = (vals[0] - vals[1]) / (2 * h)
    m.close()
    assert abs(pred) > 0
    assert abs(fd - pred) <= 2e-2 * abs(pred), (fd, pred)


@pytest.mark.parametrize("prec", [0])
def test_c3_checkpointed_matches_store_all(cuda, prec):
    torch = cuda
    from paper_2005_00281_gb300.bh import model_from_workload

    w = PRESETS["c3"](seed=0)
    nt = 1000
    w.nt = nt
    w.wavelet = np.ascontiguousarray(w.wavelet[:nt])
    src = w.shots[0]["src"][1]
    w.shots[0]["rec_iz"] = [src + 20 * k for k in range(1, 5)]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    wav = t(w.wavelet)
    out = []
    for cap in (0, 400 << 20):
        m = model_from_workload(w, checkpoint_cap_bytes=cap, snapshot_precision=prec)
        if cap:
            assert m.info("recompute_steps") > 0
        seis = m.forward(wav)
        obs = torch.zeros_like(seis)
        resid, J = m.residual_misfit(seis, obs)
        g = m.adjoint_gradient(resid)
        torch.cuda.synchronize()
        out.append((J, [x.cpu() for x in g], seis.cpu()))
        m.close()
    assert out[0][0] == out[1][0]
    assert torch.equal(out[0][2], out[1][2])
    for a, b in zip(out[0][1], out[1][1]):
        assert torch.equal(a, b)


def test_c4_subbatch_snapshot_precisions_vs_oracle(cuda, orc):
    """Two shots of the 256-shot run (their full windows, 240 rows) under a
    byte cap that forces checkpoint snapshots, shortened to 400 steps with
    the receivers moved near the source: the FP32-snapshot gradient against
    the FP64 oracle within the parity tolerance, and the BF16 / FP16
    snapshot gradients with their errors against both printed and bounded."""
    torch = cuda
    from paper_2005_00281_gb300.bh import model_from_workload

    w = PRESETS["c4"](seed=0)
    w.shots = [dict(sh) for sh in w.shots[:2]]
    w.nt = 400
    w.wavelet = np.ascontiguousarray(w.wavelet[:400])
    for sh in w.shots:
        sh["rec_iz"] = [sh["src"][1] + 20 * k for k in range(1, 5)]
    obs = np.zeros((2, 4, w.nt))
    ref = oracle_gradient(w, obs)
    grads = {}
    for prec in (0, 1, 2):
        m = model_from_workload(w, checkpoint_cap_bytes=400_000_000, snapshot_precision=prec)
        assert m.info("snapshots") >= 1 and m.info("recompute_steps") > 0
        wav = torch.from_numpy(w.wavelet).cuda()
        seis = m.forward(wav)
        resid, J = m.residual_misfit(seis, torch.zeros_like(seis))
        g = m.adjoint_gradient(resid, with_rho=False)
        torch.cuda.synchronize()
        grads[prec] = [x.cpu().numpy() for x in g[:2]]
        m.close()
    errs = {}
    for prec, name in ((0, "fp32"), (1, "bf16"), (2, "fp16")):
        errs[name] = {k: (rel_l2(grads[prec][q], ref[k]), rel_l2(grads[prec][q], grads[0][q]))
                      for q, k in enumerate(("g_lam", "g_mu"))}
    print("c4 two-shot sub-batch, rel L2 (vs oracle, vs FP32 snapshots):",
          {n: {k: tuple(f"{x:.2e}" for x in v) for k, v in e.items()} for n, e in errs.items()})
    for k in ("g_lam", "g_mu"):
        assert errs["fp32"][k][0] <= 1e-4 and errs["fp32"][k][1] == 0.0
        assert errs["fp16"][k][0] <= 5e-3 and errs["bf16"][k][0] <= 2e-2


def _bench_choice_c2(torch):
    """The launch configuration the committed autotuner cache holds for the
    64-shot logging run on this GPU: (group, form, tile code, split, order)."""
    from paper_2005_00281_gb300 import bh
    w = PRESETS["c2"](seed=0)
    P = (max(sh["nz"] for sh in w.shots) + 31) // 32 * 32
    got = bh.tune_lookup(bh.TUNE_CACHE, torch.cuda.get_device_name(0), w.nr, P, w.nshots)
    if got is None:
        pytest.skip("no committed autotuner choice for this GPU")
    return got


def test_c2_subbatch_bench_config_vs_oracle(cuda, orc):
    """Two shots of the 64-shot run (their full windows, 240 rows) in the
    launch configuration the benchmark takes from the autotuner cache (fused
    interior forward steps, per-class adjoint launches), under a byte cap
    that forces checkpoint re-runs of odd and even lengths, shortened to 400
    steps with the receivers near the source: against the FP64 oracle
    element by element."""
    torch = cuda
    from paper_2005_00281_gb300.bh import model_from_workload

    G, form, code, split, order = _bench_choice_c2(torch)
    w = PRESETS["c2"](seed=0)
    w.shots = [dict(sh) for sh in w.shots[:2]]
    w.nt = 400
    w.wavelet = np.ascontiguousarray(w.wavelet[:400])
    for sh in w.shots:
        sh["rec_iz"] = [sh["src"][1] + 20 * k for k in range(1, 5)]
    obs = np.zeros((2, 4, w.nt))
    m = model_from_workload(w, checkpoint_cap_bytes=300_000_000)
    assert m.info("recompute_steps") > 0
    m.set_option("group", min(G, 2))
    m.set_option("persistent", form)
    m.set_option("tile_code", code)
    m.set_option("split", split)
    m.set_option("tile_order", order)
    wav = torch.from_numpy(w.wavelet).cuda()
    seis = m.forward(wav)
    resid, J = m.residual_misfit(seis, torch.zeros_like(seis))
    g = m.adjoint_gradient(resid)
    H = m.hessian()
    torch.cuda.synchronize()
    gpu = dict(seis=seis.cpu().numpy(), g_lam=g[0].cpu().numpy(), g_mu=g[1].cpu().numpy(),
               g_rho=g[2].cpu().numpy(), H_lam=H[0].cpu().numpy(), H_mu=H[1].cpu().numpy())
    m.close()
    ref = oracle_gradient(w, obs)
    print("c2 two-shot sub-batch, configuration", (G, form, code, split, order))
    assert np.abs(ref["seis"]).max() > 0
    assert rel_l2(gpu["seis"], ref["seis"]) <= 1e-5
    assert abs(J - ref["J"]) <= 1e-5 * ref["J"]
    for k in ("g_lam", "g_mu", "g_rho", "H_lam", "H_mu"):
        e = rel_l2(gpu[k], ref[k])
        ea = float(np.max(np.abs(gpu[k] - ref[k])) / np.max(np.abs(ref[k])))
        print(f"  {k}: rel L2 {e:.2e}, max abs / max {ea:.2e}")
        assert e <= 1e-4 and ea <= 1e-3, (k, e, ea)


def test_c2_full_run_in_bench_config(cuda):
    """The whole 64-shot logging run (8000 steps, 240 GB checkpoint cap) in
    the benchmark's cached launch configuration, twice (the same bits), and
    once with the forward in the half-step kernels instead of the fused
    interior steps (a separately compiled path: the same misfit and
    gradients to rounding).  Every column of this model lies in the C-PML
    of some window, so a finite difference of the summed misfit is not a
    check of the per-window gradients here; the tests at small sizes and
    the two-window oracle comparison above are."""
    torch = cuda
    from paper_2005_00281_gb300.bh import TUNE_CACHE, model_from_workload

    G, form, code, split, order = _bench_choice_c2(torch)
    w = PRESETS["c2"](seed=0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    wav = t(w.wavelet)
    cap = 240 * 10**9
    truth = model_from_workload(w, checkpoint_cap_bytes=cap)
    truth.tune(cache_path=TUNE_CACHE)
    truth.set_model(t(w.vp_true), t(w.vs_true), t(w.rho_true))
    obs = truth.forward(wav).clone()
    truth.close()
    m = model_from_workload(w, checkpoint_cap_bytes=cap)
    desc = m.tune(cache_path=TUNE_CACHE)
    assert "cached" in desc
    assert (m.info("group"), m.info("tile_code"), m.info("split")) == (G, code, split)

    def run():
        seis = m.forward(wav)
        resid, J = m.residual_misfit(seis, obs)
        g = m.adjoint_gradient(resid, with_rho=False)
        torch.cuda.synchronize()
        return J, [x.cpu().numpy() for x in g[:2]]

    J1, g1 = run()
    assert m.info("recompute_steps") > 0
    J2, g2 = run()
    assert J1 == J2 and all(np.array_equal(a, b) for a, b in zip(g1, g2))
    m.set_option("split", 1)
    J3, g3 = run()
    m.close()
    errs = [rel_l2(a, b) for a, b in zip(g3, g1)]
    print(f"c2 full run, configuration {(G, form, code, split, order)}: J {J1:.9e}; "
          f"half-step forward J {J3:.9e}, gradients rel L2 {errs}")
    assert abs(J3 - J1) <= 1e-5 * abs(J1)
    assert max(errs) <= 1e-4
