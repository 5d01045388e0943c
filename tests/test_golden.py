"""Stored values under tests/golden/: the model facts the paper states
(cited there), and an oracle regression fixture written by
tests/golden/make_oracle_golden.py from the oracle alone."""
import os

import numpy as np
import pytest

from synthetic import PRESETS

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _paper_values():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_values.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                key, value, unit, *_ = line.split()
                vals[key] = (value, unit)
    return vals


@pytest.mark.parametrize("name", ["c0", "c1", "c3"])
def test_workloads_follow_the_paper_borehole(name):
    """The synthetic models put water in a borehole of the paper's radius:
    cells with centre r < radius are fluid (Vs 0), those beyond are rock."""
    vals = _paper_values()
    radius = float(vals["borehole_radius"][0])
    assert vals["borehole_radius"][1] == "m" and vals["borehole_fluid"][0] == "water"
    w = PRESETS[name]() if name == "c0" else PRESETS[name](seed=0)
    r = (np.arange(w.nr) + 0.5) * w.dr
    fluid = r < radius
    assert fluid.sum() == int(round(radius / w.dr))
    assert np.all(w.vs[fluid] == 0) and np.all(w.vs_true[fluid] == 0)
    assert np.all(w.vs[~fluid] > 0) and np.all(w.vs_true[~fluid] > 0)
    # water: P velocity 1500 m/s and density 1000 kg/m^3 (the reading of "water")
    assert np.allclose(w.vp[fluid], 1500.0) and np.allclose(w.rho[fluid], 1000.0)


def test_oracle_matches_its_stored_values(orc):
    import importlib.util

    spec = importlib.util.spec_from_file_location(
        "make_oracle_golden", os.path.join(GOLDEN, "make_oracle_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    stored = {}
    with open(os.path.join(GOLDEN, "oracle_tiny.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            key, *rest = line.split()
            stored[key] = rest
    J, seis, grads = mod.compute()
    # the oracle is FP64; other compilers contract multiply-adds differently,
    # which moves the last bits over the 300 steps
    assert J == pytest.approx(float(stored["J"][0]), rel=1e-9)
    for r, row in enumerate(seis):
        ref = np.array([float(v) for v in stored[f"seis{r}"]])
        assert np.max(np.abs(row - ref)) <= 1e-9 * np.max(np.abs(ref))
    for k, vals in grads.items():
        ref = np.array([float(v) for v in stored[k]])
        assert np.max(np.abs(np.array(vals) - ref)) <= 1e-9 * np.max(np.abs(ref)), k
