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
