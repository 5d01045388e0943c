"""Host arithmetic of bench.py's roofline (no GPU): the method's byte model
and the all-array model per cell and step, the C-PML strip fraction, the
bound label's state size, and the ncu traffic lookup that must refuse a
capture taken on other kernel sources."""
import os

import pytest

import bench
from synthetic import PRESETS


def test_method_bytes_by_hand():
    # every field read and written once per step; one shared model (m = 0)
    # or not (m = 1); strips s; the history written once and read once
    for m, shared in ((0, True), (1, False)):
        for s in (0.0, 0.25):
            for h in (0.0, 1.0):
                fv = bench.method_bytes_per_cell("fwd_vel", s, shared, h)
                fs = bench.method_bytes_per_cell("fwd_stress", s, shared, h)
                a_s = bench.method_bytes_per_cell("adj_stress", s, shared)
                a_v = bench.method_bytes_per_cell("adj_vel", s, shared)
                assert fv == 2 * 2 * 4 + 4 * m + 16 * s
                assert fs == 4 * 2 * 4 + 8 * m + 8 * h + 16 * s
                # adjoint velocities read and written, history read once,
                # three FP32 accumulators read and written, lambda and mu
                assert a_s == 16 + 8 * m + 8 + 24 + 16 * s
                assert a_v == 32 + 4 * m + 16 * s
    # a whole forward + adjoint step with history, one model: six fields
    # read and written in each direction (2 x 48), lambda, mu, rho in each
    # direction (2 x 12), the history written and read (16), three FP32
    # accumulators read and written (24)
    total = sum(bench.method_bytes_per_cell(k, 0.0, False, 1.0)
                for k in ("fwd_vel", "fwd_stress", "adj_stress", "adj_vel"))
    assert total == 2 * 48 + 2 * 12 + 16 + 24


def test_all_array_model_exceeds_the_method_model():
    for s in (0.0, 0.2):
        for k in ("fwd_vel", "fwd_stress", "adj_stress", "adj_vel"):
            assert (bench.all_array_bytes_per_cell(k, s, False, 1.0)
                    >= bench.method_bytes_per_cell(k, s, True, 1.0))
        # the fused step moves each field once per step: fewer bytes than the
        # two half-step kernels together
        assert (bench.all_array_bytes_per_cell("fwd_step", s, False, 1.0)
                < bench.all_array_bytes_per_cell("fwd_vel", s, False, 1.0)
                + bench.all_array_bytes_per_cell("fwd_stress", s, False, 1.0))
    # the density correlation adds its accumulators and v^{n-1/2}
    assert (bench.all_array_bytes_per_cell("adj_stress", 0.1, True)
            - bench.all_array_bytes_per_cell("adj_stress", 0.1, False)) == 40


def test_strip_fraction_and_state_size():
    w = PRESETS["c2"](seed=0)
    s = bench.shot_pml_fraction(w)
    lo = w.npml_r / w.nr + 2.0 * w.npml_z / max(sh["nz"] for sh in w.shots)
    hi = w.npml_r / w.nr + 2.0 * w.npml_z / min(sh["nz"] for sh in w.shots)
    assert lo <= s <= hi
    # a 32-shot group's window state is far above the 129 MB L2: the bound
    # of the batched run is HBM
    assert bench.state_bytes_per_group(w) > 10 * bench.L2_BYTES
    c1 = PRESETS["c1"](seed=0)
    assert bench.state_bytes_per_group(c1) < bench.L2_BYTES


def test_job_rate():
    # two ranks of 3e9 cell updates each in 1.5 s (the slower rank): 4 Gcell/s
    assert bench.job_rate(3e9, 2, 1500.0) == pytest.approx(4.0)


def test_traffic_lookup_refuses_other_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = "0123456789abcdef"
    monkeypatch.setattr(bench, "source_sha", lambda: sha)
    f = prof / "traffic_adj_stress_c2.txt"
    f.write_text("# comment\nkernel: adj_stress\nworkload: c2\n"
                 f"dram_bytes_per_cell_step: 111.3\nsource_sha: {sha}\n")
    assert bench.ncu_traffic("adj_stress", "c2") == pytest.approx(111.3)
    assert bench.ncu_traffic("fwd_step", "c2") is None
    f.write_text("kernel: adj_stress\nworkload: c2\n"
                 "dram_bytes_per_cell_step: 111.3\nsource_sha: ffffffffffffffff\n")
    assert bench.ncu_traffic("adj_stress", "c2") is None


def test_committed_traffic_files_name_the_current_sources():
    """Every committed traffic file bench.py reads was taken on the kernel
    sources of this tree (otherwise roofline.traffic would be null)."""
    d = os.path.join(bench.ROOT, "profiles")
    files = [f for f in os.listdir(d) if f.startswith("traffic_") and f.endswith(".txt")]
    assert files
    for f in files:
        kernel, workload = f[len("traffic_"):-len(".txt")].rsplit("_", 1)
        assert bench.ncu_traffic(kernel, workload) is not None, f
