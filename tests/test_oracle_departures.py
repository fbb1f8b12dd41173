"""Pins of the oracle's departure-time candidates (Sec. I, Sec. IV): variants of a request
departing later are tried in order and the first admissible one is kept.

The hover scenario fixes every outcome without the oracle: a known plan hovers on the
request's goal until step 300. A variant that would arrive while it hovers can capture the
goal only inside the separation cylinder of the hovering plan (or not at all within its
tight horizon), so it is rejected; a variant departing after the plan has ended flies an
empty airspace, which gives the closed-form straight track (action (0 deg, 0 m/s) every
step, capture after ceil(D / step - 1) steps) and is admitted.
"""
import math

import numpy as np
import pytest

from oracle import ADMITTED, Oracle
from paper_2008_03518_gb300 import scenarios as S

ACT15 = S.action_grid((-2.0, 0.0, 2.0))
BOX = (0.0, 0.0, 0.0, 10000.0, 10000.0, 500.0)
GOAL = (5000.0, 5000.0, 200.0)


def hover_oracle():
    o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    o.add_plan(0, np.repeat(np.array([GOAL], dtype=np.float32), 301, axis=0))  # steps 0 .. 300
    return o


def request(depart=0):
    # 3 km due east at 30 m/s: the straight track takes ceil(3000 / 30 - 1) = 99 steps
    return dict(ox=2000.0, oy=5000.0, oz=200.0, gx=GOAL[0], gy=GOAL[1], gz=GOAL[2], speed=30.0,
                depart=depart, horizon=105)


def test_first_admissible_variant_is_kept_and_has_the_straight_track():
    o = hover_oracle()
    d, tried = o.schedule_departures(request(), [0, 400, 500])
    assert d == 1 and len(tried) == 2
    assert tried[0]["verdict"] != ADMITTED and tried[1]["verdict"] == ADMITTED
    r = tried[1]
    assert r["n_points"] == 100
    assert np.all(r["actions"] == ACT15.index((0.0, 0.0)))
    k = np.arange(100, dtype=np.float64)[:, None]
    line = np.array([2000.0, 5000.0, 200.0]) + k * np.array([30.0, 0.0, 0.0])
    np.testing.assert_allclose(r["xyz"], line, atol=1e-3)
    assert o.n_plans == 2  # the hover plan and the admitted variant only


def test_rejected_variants_leave_the_table_unchanged():
    """Every variant before the chosen one has the result of scheduling it alone on the
    table as it was (rejections admit nothing), and none admitted means no change."""
    o = hover_oracle()
    d, tried = o.schedule_departures(request(), [0, 20, 60, 400])
    assert d == len(tried) - 1
    for delay, got in zip([0, 20, 60], tried[:-1]):
        alone = hover_oracle().schedule(request(delay))
        assert got["verdict"] == alone["verdict"] != ADMITTED
        np.testing.assert_array_equal(got["xyz"], alone["xyz"])
    o2 = hover_oracle()
    d2, tried2 = o2.schedule_departures(request(), [0, 10])
    assert d2 == -1 and all(t["verdict"] != ADMITTED for t in tried2)
    assert o2.n_plans == 1


def test_variants_are_taken_in_the_given_order():
    """The preferred order, not the departure time, decides: with 500 before 400 the
    variant departing at 500 is kept."""
    o = hover_oracle()
    d, tried = o.schedule_departures(request(), [0, 500, 400])
    assert d == 1
    assert math.isclose(tried[1]["xyz"][0][0], 2000.0)
