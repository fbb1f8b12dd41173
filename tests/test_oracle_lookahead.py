"""Pins of the oracle's lookahead window W (Sec. IV "Forward project": each action is held
for W sub-steps of dt; Alg. 9: the action's value is the largest value along them).

Closed forms and brute force with library trigonometry, independent of the oracle's code:
- goal only: the value of an action is r * gamma^(least goal distance of its W projected
  states), and the chosen action the one whose projection passes closest to the goal;
- a moving plan: projected state j is scored against the plan's sample at t + j with the
  plan's velocity from t + j to t + j + 1 (a wrong time index gives another value);
- projected states outside the box do not count, but the action stays valid while x_1 is
  inside;
- with nothing but the goal on the track, W > 1 flies the same straight track as W = 1.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2008_03518_gb300 import scenarios as S

ACT15 = S.action_grid((-2.0, 0.0, 2.0))
BOX = (0.0, 0.0, 0.0, 10000.0, 10000.0, 500.0)


def req(ox, oy, oz, gx, gy, gz, speed=30.0, depart=0, horizon=600):
    return dict(ox=ox, oy=oy, oz=oz, gx=gx, gy=gy, gz=gz, speed=speed, depart=depart, horizon=horizon)


@pytest.mark.parametrize("W", [2, 5, 10])
def test_goal_only_value_is_the_nearest_projected_state(W):
    o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0), lookahead_W=W)
    rng = np.random.default_rng(17 + W)
    for _ in range(60):
        s = np.array([*rng.uniform(2000, 8000, 2), rng.uniform(150, 350)])
        org = rng.uniform(0, 10000, 2)
        goal = np.array([*rng.uniform(0, 10000, 2), rng.uniform(50, 450)])
        h = int(rng.integers(0, 24))
        sp = rng.uniform(20, 40)
        q = o.q_values(s, h, 0, sp, origin=org, goal=goal)
        psi0 = math.atan2(goal[1] - org[1], goal[0] - org[0])
        best = []
        for a, (dpsi, climb) in enumerate(ACT15):
            psi = psi0 + math.radians(15.0 * h + dpsi)
            step = np.array([sp * math.cos(psi), sp * math.sin(psi), climb])
            d = min(np.linalg.norm(goal - (s + j * step)) for j in range(1, W + 1))
            assert q["Q"][a] == pytest.approx(200.0 * 0.99 ** d, rel=1e-9)
            assert q["nxt"][a] == pytest.approx(s + step, abs=1e-9)  # the move is one sub-step
            best.append(d)
        srt = np.sort(best)
        if srt[1] - srt[0] > 1e-6:
            assert int(np.argmax(q["Q"])) == int(np.argmin(best))


def _line_plan(v, n=100, z=200.0):
    """Plan along +x moving v metres per step, from x = 0 at step 0."""
    x = v * np.arange(n, dtype=np.float64)
    return np.stack([x, np.zeros(n), np.full(n, z)], axis=1).astype(np.float32)


def test_projected_states_use_the_plan_at_their_own_step():
    """A plan moves +x at 20 m/step. Scoring at t = 10 with W = 3, an action moving +x at
    30 m/step from x = 450 projects x_j = 450 + 30 j, to be scored against the wells
    centred at p(10 + j) + tau * 20 = 200 + 20 j + 20 tau (radius 300 + 10 tau). With
    goal_reward 0 and MAX, the value of x_j is minus the largest 1000 * .97^d over the wells
    it is inside, and the action's value the largest of the three; written out below."""
    o = Oracle(BOX, 1.0, 0.99, [(0.0, 0.0)], (150.0, 30.0), goal_reward=0.0, lookahead_W=3)
    o.add_plan(0, _line_plan(20.0))
    q = o.q_values([450.0, 0.0, 200.0], 0, 10, 30.0, origin=[0.0, 0.0], goal=[9000.0, 0.0, 200.0])
    taus = (-5.0, 0.0, 5.0, 10.0, 15.0)
    vals = []
    for j in (1, 2, 3):
        x = 450.0 + 30.0 * j
        pen = 0.0
        for tau in taus:
            c = 20.0 * (10 + j) + tau * 20.0
            d = abs(x - c)
            if d < 300.0 + 10.0 * tau:
                pen = max(pen, 1000.0 * 0.97 ** d)
        vals.append(-pen)
    assert q["Q"][0] == pytest.approx(max(vals), rel=1e-12)
    # the same state scored one step later (t = 11) gives another value: the index matters
    q2 = o.q_values([450.0, 0.0, 200.0], 0, 11, 30.0, origin=[0.0, 0.0], goal=[9000.0, 0.0, 200.0])
    assert q2["Q"][0] != pytest.approx(q["Q"][0], rel=1e-6)


def test_projected_states_outside_the_box_do_not_count():
    """x = 940 heading +x at 30 m/step in a box ending at x = 1000: x_1 = 970 and x_2 = 1000
    are inside (the box is closed), x_3 = 1030 is not. The goal lies beyond the edge, so
    the value grows with j and stops at x_2."""
    box = (0.0, 0.0, 0.0, 1000.0, 1000.0, 500.0)
    o = Oracle(box, 1.0, 0.99, [(0.0, 0.0)], (150.0, 30.0), lookahead_W=3)
    q = o.q_values([940.0, 500.0, 200.0], 0, 0, 30.0, origin=[0.0, 500.0], goal=[1100.0, 500.0, 200.0])
    assert q["valid"][0]
    assert q["Q"][0] == pytest.approx(200.0 * 0.99 ** 100.0, rel=1e-12)
    # starting 30 m further, x_1 = 1000 is the last state inside
    q = o.q_values([970.0, 500.0, 200.0], 0, 0, 30.0, origin=[0.0, 500.0], goal=[1100.0, 500.0, 200.0])
    assert q["valid"][0] and q["Q"][0] == pytest.approx(200.0 * 0.99 ** 100.0, rel=1e-12)
    q = o.q_values([980.0, 500.0, 200.0], 0, 0, 30.0, origin=[0.0, 500.0], goal=[1100.0, 500.0, 200.0])
    assert not q["valid"][0]


def test_straight_track_is_the_same_for_every_window():
    rng = np.random.default_rng(3)
    o1 = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    for W in (3, 10):
        oW = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0), lookahead_W=W)
        for _ in range(5):
            ox, oy, gx, gy = rng.uniform(1000, 9000, 4)
            z = rng.uniform(100, 400)
            r = req(ox, oy, z, gx, gy, z, speed=rng.uniform(20, 40), horizon=2000)
            a, b = o1.rollout(r), oW.rollout(r)
            assert a["n_points"] == b["n_points"]
            np.testing.assert_array_equal(a["xyz"], b["xyz"])
