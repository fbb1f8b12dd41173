"""Pins of the oracle's batch co-simulation (Alg. 1 "DistributedUam" with the batch's
aircraft as each other's Table 3 wells; Sec. V, aircraft of a batch that may meet).

- one request alone, or requests too far apart to reach each other's wells, fly exactly
  their solo rollouts (the other aircraft add nothing outside the wells' radii);
- the wells of another aircraft sit at its position at t plus tau times its last move over
  dt, with radii 300 + 10 tau: the values of a step are written out here from that rule;
- two aircraft flying head-on along one line meet when each is planned alone against an
  empty table, and keep separation when co-simulated.
"""
import math

import numpy as np
import pytest

from oracle import ADMITTED, Oracle
from paper_2008_03518_gb300 import scenarios as S

ACT15 = S.action_grid((-2.0, 0.0, 2.0))
BOX = (0.0, 0.0, 0.0, 10000.0, 10000.0, 500.0)


def req(ox, oy, oz, gx, gy, gz, speed=30.0, depart=0, horizon=600):
    return dict(ox=ox, oy=oy, oz=oz, gx=gx, gy=gy, gz=gz, speed=speed, depart=depart, horizon=horizon)


def test_single_and_distant_requests_fly_their_solo_rollouts():
    o = Oracle.from_scenario(S.c1_plain_small())
    a = req(1000.0, 1000.0, 200.0, 4000.0, 1500.0, 250.0)
    b = req(9000.0, 9000.0, 300.0, 6000.0, 8500.0, 200.0, depart=5)  # kilometres away throughout
    for batch in ([a], [a, b]):
        co = o.cosim(batch)
        for r, d in zip(batch, co):
            solo = o.rollout(r)
            assert d["n_points"] == solo["n_points"]
            np.testing.assert_array_equal(d["xyz"], solo["xyz"])
            np.testing.assert_array_equal(d["actions"], solo["actions"])


def test_other_aircraft_wells_at_position_plus_tau_times_last_move():
    """Aircraft 1 flies +x from (1000, 0, 200) at 30 m/s; aircraft 0 starts 474 m away, out
    of every well of aircraft 1 at step 0 (velocity 0 then, all centres at its origin).
    At step 1 aircraft 1 is at (1030, 0, 200) with velocity (30, 0, 0): its wells sit at
    x = 1030 + 30 tau, tau = -5 .. 15, radii 250 .. 450. Aircraft 0's action values at step
    1 are its goal term minus the largest 1000 * .97^d of those wells it is inside."""
    o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    r0 = req(1480.0, 150.0, 200.0, 1480.0, 3000.0, 200.0)   # heads +y
    r1 = req(1000.0, 0.0, 200.0, 8000.0, 0.0, 200.0)        # heads +x
    co = o.cosim([r0, r1], trace=True)
    straight = ACT15.index((0.0, 0.0))
    assert co[0]["actions"][0] == straight and co[1]["actions"][0] == straight
    s0 = np.array([1480.0, 180.0, 200.0])
    np.testing.assert_allclose(co[0]["xyz"][1], s0, atol=1e-4)
    goal = np.array([1480.0, 3000.0, 200.0])
    for a, (dpsi, climb) in enumerate(ACT15):
        psi = math.pi / 2 + math.radians(dpsi)
        nx = s0 + np.array([30.0 * math.cos(psi), 30.0 * math.sin(psi), climb])
        pen = 0.0
        for tau in (-5.0, 0.0, 5.0, 10.0, 15.0):
            c = np.array([1030.0 + 30.0 * tau, 0.0, 200.0])
            d = np.linalg.norm(nx - c)
            if d < 300.0 + 10.0 * tau:
                pen = max(pen, 1000.0 * 0.97 ** d)
        want = 200.0 * 0.99 ** np.linalg.norm(goal - nx) - pen
        assert co[0]["q"][1][a] == pytest.approx(want, rel=1e-9, abs=1e-9)


def test_head_on_pair_collides_alone_and_separates_when_co_simulated():
    a = req(2000.0, 5000.0, 200.0, 8000.0, 5000.0, 200.0, horizon=400)
    b = req(8000.0, 5000.0, 200.0, 2000.0, 5000.0, 200.0, horizon=400)
    o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    ra, rb = o.rollout(a), o.rollout(b)
    n = min(ra["n_points"], rb["n_points"])
    gap = np.hypot(*(ra["xyz"][:n, :2] - rb["xyz"][:n, :2]).T)
    assert gap.min() < 150.0  # straight lines meet
    o2 = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    out = o2.schedule_cosim([a, b])
    assert [d["verdict"] for d in out] == [ADMITTED, ADMITTED]
    n = min(out[0]["n_points"], out[1]["n_points"])
    pa, pb = out[0]["xyz"][:n], out[1]["xyz"][:n]
    conflict = (np.hypot(*(pa[:, :2] - pb[:, :2]).T) < 150.0) & (np.abs(pa[:, 2] - pb[:, 2]) < 30.0)
    assert not conflict.any()
    # admitting the straight tracks one after the other instead: the second conflicts
    o3 = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    o3.add_plan(0, ra["xyz"])
    assert o3.sep_check(0, rb["xyz"])["first_conflict"] >= 0
