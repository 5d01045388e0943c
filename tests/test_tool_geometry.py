"""The multi-source logging tool of the Numerical Examples (Fig. 2): the
raw acquisition table, its realignment to one source and 39 receivers, and
the batched workload built on it.  Geometry only (no GPU)."""
import numpy as np
import pytest

from synthetic.workloads import (FT, STATION, TOOL_SOURCES, TOOL_STATIONS, realign,
                                 tool_logging_run, tool_records)
from tests.test_golden import _paper_values


def test_tool_follows_the_paper():
    vals = _paper_values()
    assert int(vals["receiver_stations"][0]) == TOOL_STATIONS
    assert vals["receiver_spacing"][1] == "ft" and vals["logging_step"][1] == "ft"
    assert STATION == pytest.approx(float(vals["receiver_spacing"][0]) * FT)
    assert int(vals["modelled_monopoles"][0]) == len(TOOL_SOURCES)
    assert int(vals["realigned_receivers"][0]) == len(TOOL_SOURCES) * TOOL_STATIONS
    recs = tool_records(3, 5.0)
    # three records per tool depth, 13 receivers 0.5 ft apart, the tool moves 0.5 ft
    assert len(recs) == 9
    for r in recs:
        assert np.allclose(np.diff(r["z_rec"]), -STATION)
    assert recs[3]["z_src"] - recs[0]["z_src"] == pytest.approx(
        float(vals["logging_step"][0]) * FT)


def test_realignment_gives_39_consecutive_receivers():
    near = 3.0
    recs = tool_records(60, 12.0, near_offset=near)
    gathers = realign(recs)
    # every source depth that all three monopoles visit: 60 - 2 * 13 of them
    assert len(gathers) == 60 - 2 * TOOL_STATIONS
    used = set()
    for zs, rows in gathers.items():
        offs = np.array([o for o, _, _ in rows])
        assert len(rows) == 39
        np.testing.assert_allclose(offs, near + STATION * np.arange(39), atol=1e-9)
        # the three monopoles' arrays, nearest first
        names = [recs[i]["source"] for _, i, _ in rows]
        assert names == [n for n in TOOL_SOURCES for _ in range(TOOL_STATIONS)]
        for _, i, q in rows:
            assert (i, q) not in used
            used.add((i, q))
            assert recs[i]["z_src"] == pytest.approx(zs)
    # each raw receiver record of a realigned source depth is used exactly once
    for i, r in enumerate(recs):
        if any(abs(r["z_src"] - zs) < 1e-9 for zs in gathers):
            assert all((i, q) in used for q in range(TOOL_STATIONS))


def test_tool_workload_windows():
    w = tool_logging_run(ndepths=6, nt=100)
    assert w.nshots == 6
    for k, sh in enumerate(w.shots):
        assert len(sh["rec_iz"]) == 39
        assert w.npml_z <= min(sh["rec_iz"]) and max(sh["rec_iz"]) < sh["nz"] - w.npml_z
        assert w.npml_z <= sh["src"][1] < sh["nz"] - w.npml_z
        assert sh["z_offset"] >= 0 and sh["z_offset"] + sh["nz"] <= w.nz
        # receivers 0.5 ft apart on the grid (rounded to the nearest cell)
        offs = (sh["src"][1] - np.array(sh["rec_iz"])[::-1]) * w.dz
        # source and receiver each rounded to the nearest cell
        np.testing.assert_allclose(offs, 3.0 + STATION * np.arange(39), atol=w.dz + 1e-9)
        if k:
            step = (sh["z_offset"] + sh["src"][1]) - (w.shots[k - 1]["z_offset"] +
                                                      w.shots[k - 1]["src"][1])
            assert abs(step * w.dz - STATION) <= w.dz
