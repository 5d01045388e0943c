"""Host logic of the binomial checkpoint schedule (no GPU): the plan that the
library executes reverses every segment exactly once, in reverse order, each
from the right forward state, within the binomial repetition bound."""
import math

import pytest

ADVANCE, TAKE, RESTORE, REVERSE = 0, 1, 2, 3


@pytest.fixture(scope="module")
def plan():
    import shutil
    import os
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2005_00281_gb300.build import build_library
    build_library()
    from paper_2005_00281_gb300 import bh
    return bh.checkpoint_plan


def simulate(nseg, nsnap, spine, actions):
    """Run the plan on a symbolic forward state; returns (advanced segments,
    reversal order).  Fails on any inconsistency."""
    slots = {0: 0}  # slot -> segment whose state it holds
    pos = 0
    for seg, slot in spine:             # the forward sweep takes these on the way
        assert seg > pos and 1 <= slot <= nsnap and slot not in slots
        pos = seg
        slots[slot] = seg
    cur = None                          # segment of the current forward state
    advanced = 0
    order = []
    live = set(slots)
    for kind, a, b in actions:
        if kind == RESTORE:
            assert a in slots and slots[a] == b, (a, b, slots)
            cur = b
        elif kind == ADVANCE:
            assert cur == a and b > a
            advanced += b - a
            cur = b
        elif kind == TAKE:
            assert cur == b and 1 <= a <= nsnap
            slots[a] = b
        elif kind == REVERSE:
            assert cur == a
            order.append(a)
            cur = None                  # the state moved on while refilling the window
        else:
            raise AssertionError(kind)
    assert live  # slot 0 always exists
    return advanced, order


@pytest.mark.parametrize("nseg,nsnap", [(1, 0), (2, 0), (7, 0), (10, 1), (10, 2), (37, 3),
                                        (100, 5), (250, 10), (1000, 20), (64, 63)])
def test_plan_reverses_every_segment_once(plan, nseg, nsnap):
    spine, actions = plan(nseg, nsnap)
    advanced, order = simulate(nseg, nsnap, spine, actions)
    assert order == list(range(nseg - 1, -1, -1))
    # binomial bound: with t the least repetition number, C(s + t, s) >= n,
    # no segment is advanced more than t times (the sweep counts once)
    if nsnap > 0:
        t = 1
        while math.comb(nsnap + t, nsnap) < nseg:
            t += 1
        assert advanced + nseg <= t * nseg
    else:
        assert advanced == nseg * (nseg - 1) // 2


def test_enough_slots_cost_nothing(plan):
    # with a slot for every segment boundary the sweep takes them all and
    # the reversal only restores
    spine, actions = plan(16, 15)
    advanced, _ = simulate(16, 15, spine, actions)
    assert advanced == 0 and len(spine) == 15


@pytest.fixture(scope="module")
def plan_history():
    import shutil
    import os
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2005_00281_gb300.build import build_library
    build_library()
    from paper_2005_00281_gb300 import bh
    return bh.plan_history


def _bytes(nt, h, S, L, s, tail):
    if tail >= nt:
        return (nt + 1) * h
    return (max(tail, L) + 1) * h + s * S


def test_history_plan_stores_everything_when_it_fits(plan_history):
    assert plan_history(100, 10.0, 70.0, 101 * 10) == (100, 0, 100, 0)


@pytest.mark.parametrize("nt,h,S", [(60, 10.0, 70.0), (97, 3.0, 40.0), (40, 5.0, 12.0)])
def test_history_plan_matches_brute_force(plan_history, nt, h, S):
    """Over every cap from one window to everything stored: the plan fits
    the cap, and whenever a plan with a tail and a snapshot at every earlier
    segment fits, its recompute is the least any such plan has (brute force
    over every L and segment count); more memory never costs recompute."""
    last = None
    for cap in range(int(2 * h), int((nt + 2) * h), max(1, int(h // 2))):
        try:
            L, s, tail, rec = plan_history(nt, h, S, cap)
        except Exception:
            continue
        assert _bytes(nt, h, S, L, s, tail) <= cap
        best = None
        for LL in range(1, nt):
            nseg = -(-nt // LL)
            for nsp in range(1, nseg):
                t = nt - nsp * LL
                if (max(t, LL) + 1) * h + (nsp - 1) * S <= cap:
                    best = nsp * LL if best is None else min(best, nsp * LL)
        if (nt + 1) * h <= cap:
            best = 0
        if best is not None:
            assert rec == best, (cap, rec, best)
            assert rec == (nt - tail if tail < nt else 0)
        else:
            assert tail == 0 and rec >= nt
        if last is not None:
            assert rec <= last
        last = rec


def test_history_plan_batched_logging_run(plan_history):
    """The 64-shot logging run (windows padded to 2016 cells by 240, 8000
    steps) under a 200 GB and a 240 GB cap: the sweep keeps a tail, and only
    the steps before it are re-run (0.91 and 0.89 of nt), where a
    window-only plan re-runs every step."""
    h = 2 * 64 * 240 * 2016 * 4.0
    S = 14 * 64 * 240 * 2016 * 4.0
    for cap, bound in ((200e9, 0.91), (240e9, 0.89)):
        L, s, tail, rec = plan_history(8000, h, S, cap)
        assert tail > 0 and rec == 8000 - tail and rec < bound * 8000, (cap, rec)
        assert _bytes(8000, h, S, L, s, tail) <= cap
