"""Pins of the FP64 CPU oracle against facts that do not come from the oracle itself.

Each test ties one part of the oracle to a value the paper prints, a closed-form
geometry, a library routine, brute force on a tiny input, or an invariant of the
method, so that a dropped term, a flipped sign, a wrong time index or a transposed
operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import (ADMITTED, PAPER_WELLS, REJ_CONFLICT, REJ_HORIZON, REJ_NO_ACTION, Oracle,
                    heading_table)
from paper_2008_03518_gb300 import scenarios as S

pytestmark = pytest.mark.filterwarnings("ignore")

ACT15 = S.action_grid((-2.0, 0.0, 2.0))
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_rows(name):
    """Rows of a fixture under tests/golden (whitespace-separated, '#' comments)."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows
BOX = (0.0, 0.0, 0.0, 10000.0, 10000.0, 500.0)


def req(ox, oy, oz, gx, gy, gz, speed=30.0, depart=0, horizon=600):
    return dict(ox=ox, oy=oy, oz=oz, gx=gx, gy=gy, gz=gz, speed=speed, depart=depart, horizon=horizon)


# ---------------------------------------------------------------- Fig. 2a, Table 3


def test_fig2a_risk_well_values():
    """Fig. 2 plots the truncated risk well -2 * 0.7^|x-5| for 2 < x < 8 and 0 outside
    (tests/golden/fig2_risk_well.txt).

    A single static well {r=-2, gamma=.7, p=(5,0,0), R=3} and no goal reward must give
    exactly that curve as the value of a successor at (x, 0, 0)."""
    (mag, dec, ctr, rad), = [list(map(float, r)) for r in golden_rows("fig2_risk_well.txt")]
    o = Oracle((-100, -100, -100, 100, 100, 100), 1.0, 0.99, [(0.0, 0.0)], (1.0, 1.0), wells=(),
               goal_reward=0.0, static_wells=np.array([[ctr, 0.0, 0.0, rad, mag, dec]]))
    for x in (-1.0, 2.0, 2.0 + 1e-9, 2.5, 3.0, 4.2, 5.0, 5.5, 7.0, 7.999, 8.0, 9.5):
        # state one metre behind x, moving +x at 1 m/s: the only successor is (x, 0, 0)
        q = o.q_values([x - 1.0, 0.0, 0.0], 0, 0, 1.0, origin=[0.0, 0.0], goal=[1.0e3, 0.0, 0.0])
        expect = -mag * dec ** abs(x - ctr) if ctr - rad < x < ctr + rad else 0.0
        assert q["valid"][0]
        assert q["Q"][0] == pytest.approx(expect, rel=1e-12, abs=1e-300), x


def test_table3_default_wells():
    """Table 3, intruder row: magnitude -1000, decay .97, location p + v t, radius 300 + 10 t,
    t in {-5, 0, 5, 10, 15} (tests/golden/table3_intruder_wells.txt)."""
    rows = tuple(tuple(map(float, r)) for r in golden_rows("table3_intruder_wells.txt"))
    assert len(rows) == 5
    for t, radius, _, _ in rows:
        assert radius == 300.0 + 10.0 * t
    assert PAPER_WELLS == rows


def _line_plan(v_before, v_after, k_switch=50, n=100, z=200.0):
    """Plan along +x whose per-step displacement changes from v_before to v_after after k_switch."""
    x = np.zeros(n)
    for k in range(1, n):
        x[k] = x[k - 1] + (v_before if k <= k_switch else v_after)
    return np.stack([x, np.zeros(n), np.full(n, z)], axis=1).astype(np.float32)


@pytest.mark.parametrize("combine", [0, 1])
@pytest.mark.parametrize("dt", [1.0, 0.5])
def test_moving_plan_wells_time_index_velocity_and_sign(combine, dt):
    """Wells sit at p(t+1) + tau * v with v = p(t+2) - p(t+1) (the plan's own next
    displacement), evaluated for a successor at time t+1.

    The plan moves 20 m/step until step 50, then 40 m/step. Scoring at t = 49 uses
    p(50) = 1000 and v = 40, so the wells are centred at 800, 1000, 1200, 1400, 1600 with
    radii 250..450. A successor at x = 1700 is 100 m from the tau=15 well (R 450) and
    300 m from the tau=10 well (R 400), outside the others. Using p(t), a backward
    velocity or wells behind the plan all give different penalties. At dt = 0.5 s the
    velocity doubles (80 m/s), the wells move to 600..2200 and the successor is inside
    the tau=10 (100 m) and tau=5 (300 m) wells: the same two values."""
    o = Oracle(BOX, dt, 0.99, [(0.0, 0.0)], (150.0, 30.0), combine=combine, goal_reward=0.0)
    o.add_plan(0, _line_plan(20.0, 40.0))
    q = o.q_values([1690.0, 0.0, 200.0], 0, 49, 10.0 / dt, origin=[0.0, 0.0], goal=[5000.0, 0.0, 200.0])
    a, b = 1000.0 * 0.97 ** 100.0, 1000.0 * 0.97 ** 300.0
    expect = (a + b) if combine else a
    assert q["P"][0] == pytest.approx(expect, rel=1e-12)
    assert q["Q"][0] == pytest.approx(-expect, rel=1e-12)


def test_plan_ending_has_zero_velocity():
    """A plan with no sample at t+2 has no velocity: all five wells share its last point,
    so a successor 440 m away lies only inside the R = 450 well."""
    o = Oracle(BOX, 1.0, 0.99, [(0.0, 0.0)], (150.0, 30.0), goal_reward=0.0)
    pts = np.array([[1000.0, 0.0, 200.0], [1000.0, 0.0, 200.0]], dtype=np.float32)
    o.add_plan(9, pts)  # present at 9 and 10 only
    q = o.q_values([1430.0, 0.0, 200.0], 0, 9, 10.0, origin=[0, 0], goal=[9000.0, 0.0, 200.0])
    assert q["P"][0] == pytest.approx(1000.0 * 0.97 ** 440.0, rel=1e-12)
    # at t = 10 the plan has no sample at t+1 = 11: no penalty at all
    q = o.q_values([1430.0, 0.0, 200.0], 0, 10, 10.0, origin=[0, 0], goal=[9000.0, 0.0, 200.0])
    assert q["P"][0] == 0.0


def test_classes_are_combined_by_max():
    """Alg. 8: V = V+ - max(V-, V^T, V^I) - V_alt: a static (terrain) well and a plan well
    overlap; MAX keeps the larger, SUM adds them."""
    sw = np.array([[1500.0, 0.0, 200.0, 500.0, 1000.0, 0.99]])
    for combine in (0, 1):
        o = Oracle(BOX, 1.0, 0.99, [(0.0, 0.0)], (150.0, 30.0), goal_reward=0.0, static_wells=sw,
                   combine=combine)
        o.add_plan(0, np.tile(np.array([[1200.0, 0.0, 200.0]], dtype=np.float32), (20, 1)))
        q = o.q_values([1290.0, 0.0, 200.0], 0, 5, 10.0, origin=[0, 0], goal=[9000.0, 0.0, 200.0])
        well = 1000.0 * 0.97 ** 100.0  # plan at 1200, v = 0: d = 100, inside all five wells
        terr = 1000.0 * 0.99 ** 200.0  # static well at 1500: d = 200 < 500
        assert q["P"][0] == pytest.approx(5 * well + terr if combine else max(well, terr), rel=1e-12)


def test_work_count_matches_table2_formula():
    """Table 2 counts 5 x N x A x R_i intruder-reward threads (13,500,000 at A = 1350,
    R_i = 2000): every (action, intruder, well) triple is evaluated once per step. The
    printed sample sizes (tests/golden/table1_table2_sizes.txt) follow from the same
    counts: 5 wells of 6 FP64 fields per intruder, W projected states of 12 fields per
    action."""
    g = {k: int(v) for k, v in golden_rows("table1_table2_sizes.txt")}
    N, A, Rt, Ri, W = g["N"], g["A"], g["R_t"], g["R_i"], g["W"]
    assert g["table2_intruder_threads"] == len(PAPER_WELLS) * N * A * Ri
    assert g["table2_terrain_threads"] == N * A * Rt
    assert g["table2_forward_project_threads"] == N * A
    assert g["table1_P_I_bytes"] == len(PAPER_WELLS) * Ri * 6 * 8
    assert g["table1_P_T_bytes"] == Rt * 6 * 8
    assert g["table1_Delta10_bytes"] == N * A * W * 12 * 8
    assert g["table1_V_bytes"] == N * A * W * 8
    rng = np.random.default_rng(3)
    o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    for _ in range(37):
        o.add_plan(0, rng.uniform(0, 500, size=(50, 3)).astype(np.float32))
    for _ in range(5):
        o.add_plan(100, rng.uniform(0, 500, size=(50, 3)).astype(np.float32))  # absent at t+1
    q = o.q_values([5000.0, 5000.0, 250.0], 0, 10, 30.0, origin=[0, 0], goal=[1, 1, 250.0])
    assert q["tests"] == 5 * len(ACT15) * 37


# ---------------------------------------------------------------- geometry and goal


def test_heading_table_matches_library_trig():
    rng = np.random.default_rng(7)
    for _ in range(50):
        ox, oy, gx, gy = rng.uniform(-1e4, 1e4, 4)
        C, S_ = heading_table(ox, oy, gx, gy)
        psi0 = math.atan2(gy - oy, gx - ox)
        k = np.arange(24)
        np.testing.assert_allclose(C, np.cos(psi0 + k * np.pi / 12), atol=4e-16)
        np.testing.assert_allclose(S_, np.sin(psi0 + k * np.pi / 12), atol=4e-16)
    C, S_ = heading_table(5.0, 5.0, 5.0, 5.0)  # coincident: bearing 0
    assert C[0] == 1.0 and S_[0] == 0.0 and C[6] == 0.0 and S_[6] == 1.0


@pytest.mark.parametrize("dt", [1.0, 0.1])
def test_goal_peak_closed_form(dt):
    """Alg. 4: the goal contributes |r| gamma^d with d the successor's distance to the goal.
    Successors computed here with library cos/sin for a +x bearing; dt = 0.1 s is the
    paper's own step (Sec. IV, forward projection)."""
    o = Oracle(BOX, dt, 0.99, ACT15, (150.0, 30.0), goal_reward=200.0)
    s = np.array([1000.0, 2000.0, 100.0])
    goal = np.array([4000.0, 2000.0, 130.0])
    q = o.q_values(s, 0, 0, 25.0, origin=s[:2], goal=goal)
    for a, (dpsi, climb) in enumerate(ACT15):
        nx = s + dt * np.array([25.0 * math.cos(math.radians(dpsi)), 25.0 * math.sin(math.radians(dpsi)), climb])
        d = np.linalg.norm(goal - nx)
        assert q["nxt"][a] == pytest.approx(nx, abs=1e-9)
        assert q["Q"][a] == pytest.approx(200.0 * 0.99 ** d, rel=1e-12)


def test_empty_airspace_straight_track():
    """With no peaks but the goal and the goal at the origin's altitude, the greedy policy
    flies the bearing: action (0 deg, 0 m/s) every step, points on the straight line,
    and capture after ceil(D / step - 1) steps."""
    o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    straight = ACT15.index((0.0, 0.0))
    rng = np.random.default_rng(11)
    for _ in range(20):
        ox, oy, gx, gy = rng.uniform(500, 9500, 4)
        z = rng.uniform(50, 450)
        sp = rng.uniform(20, 40)
        D = math.hypot(gx - ox, gy - oy)
        if abs(D / sp - round(D / sp)) < 1e-6:
            continue
        d = o.rollout(req(ox, oy, z, gx, gy, z, speed=sp, horizon=2000))
        steps = max(0, math.ceil(D / sp - 1.0))
        assert d["verdict"] == -1 or d["captured"]
        assert d["n_points"] == steps + 1
        assert np.all(d["actions"] == straight)
        k = np.arange(d["n_points"])[:, None]
        line = np.array([ox, oy, z]) + k * sp * np.array([(gx - ox) / D, (gy - oy) / D, 0.0])
        np.testing.assert_allclose(d["states"], line, atol=1e-6)


def test_only_goal_argmax_is_nearest_successor():
    """With the goal as the only peak, the chosen action is the successor nearest to the
    goal; successors enumerated here by brute force with library trig."""
    o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    rng = np.random.default_rng(5)
    for _ in range(200):
        s = np.array([*rng.uniform(1000, 9000, 2), rng.uniform(100, 400)])
        org = rng.uniform(0, 10000, 2)
        goal = np.array([*rng.uniform(0, 10000, 2), rng.uniform(50, 450)])
        h = int(rng.integers(0, 24))
        sp = rng.uniform(20, 40)
        q = o.q_values(s, h, 0, sp, origin=org, goal=goal)
        psi0 = math.atan2(goal[1] - org[1], goal[0] - org[0])
        dist = []
        for dpsi, climb in ACT15:
            psi = psi0 + math.radians(15.0 * h + dpsi)
            nx = s + np.array([sp * math.cos(psi), sp * math.sin(psi), climb])
            dist.append(np.linalg.norm(goal - nx))
        dist = np.array(dist)
        srt = np.sort(dist)
        if srt[1] - srt[0] < 1e-6:
            continue
        assert int(np.argmax(q["Q"])) == int(np.argmin(dist))


# ---------------------------------------------------------------- terrain and hard deck


def test_terrain_bilinear_matches_scipy():
    from scipy.interpolate import RegularGridInterpolator
    rng = np.random.default_rng(2)
    hm = rng.uniform(0, 300, size=(33, 41)).astype(np.float32)
    box = (100.0, -200.0, 0.0, 4100.0, 3000.0, 1000.0)
    o = Oracle(box, 1.0, 0.99, ACT15, (150.0, 30.0), heightmap=hm, clearance=60.0)
    xs = np.linspace(box[0], box[3], hm.shape[1])
    ys = np.linspace(box[1], box[4], hm.shape[0])
    f = RegularGridInterpolator((ys, xs), hm.astype(np.float64), method="linear")
    for x, y in rng.uniform([box[0], box[1]], [box[3], box[4]], size=(300, 2)):
        assert o.terrain(x, y) == pytest.approx(float(f([[y, x]])[0]), abs=1e-9)
    assert o.terrain(box[3], box[4]) == pytest.approx(float(hm[-1, -1]), abs=1e-9)


def test_hard_deck_penalty_on_flat_terrain():
    """Alg. 1 hard deck, 1000 - altitude below the penalty altitude, read as clearance
    over terrain: flat terrain at 100 m and a 60 m clearance."""
    hm = np.full((5, 5), 100.0, dtype=np.float32)
    o = Oracle(BOX, 1.0, 0.99, [(0.0, 0.0)], (150.0, 30.0), heightmap=hm, clearance=60.0, goal_reward=0.0)
    for z, expect in ((130.0, 970.0), (160.0, 0.0), (159.5, 940.5), (90.0, 1010.0)):
        q = o.q_values([4990.0, 5000.0, z], 0, 0, 10.0, origin=[0, 5000.0], goal=[9000.0, 5000.0, z])
        assert q["V"][0] == pytest.approx(expect, abs=1e-9)
        assert q["Q"][0] == pytest.approx(-expect, abs=1e-9)


# ---------------------------------------------------------------- separation check


def test_sep_check_crossing_geometry():
    """Two straight tracks through the same point at the same step: strict minima, so
    exactly 150 m / 30 m apart is separated and anything less is a conflict."""
    o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    n = 41
    k = np.arange(n, dtype=np.float64)
    known = np.stack([1500.0 + 200.0 * (k - 20.0), np.full(n, 5000.0), np.full(n, 200.0)], 1).astype(np.float32)
    o.add_plan(10, known)  # at (1500, 5000, 200) at step 30; 200 m/step so only that step is close
    for dy, dz, conflict in ((0.0, 0.0, True), (149.75, 0.0, True), (150.0, 0.0, False),
                             (0.0, 29.5, True), (0.0, 30.0, False), (100.0, 20.0, True),
                             (120.0, 0.0, True), (0.0, -30.0, False)):
        traj = np.stack([np.full(n, 1500.0), 5000.0 + dy + 200.0 * (k - 20.0), np.full(n, 200.0 + dz)],
                        1).astype(np.float32)  # crosses the known plan at step 20 (t = 30)
        r = o.sep_check(10, traj)
        if conflict:
            assert r["first_conflict"] == 20 and r["conflicts"] >= 1, (dy, dz)
        else:
            assert r["first_conflict"] == -1 and r["conflicts"] == 0, (dy, dz)


def test_sep_check_matches_cdist_bruteforce():
    from scipy.spatial.distance import cdist
    rng = np.random.default_rng(9)
    for trial in range(30):
        o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
        plans = []
        for _ in range(5):
            t0 = int(rng.integers(0, 10))
            xyz = rng.uniform([0, 0, 0], [400, 400, 60], size=(int(rng.integers(1, 20)), 3)).astype(np.float32)
            o.add_plan(t0, xyz)
            plans.append((t0, xyz))
        t0 = int(rng.integers(0, 10))
        traj = rng.uniform([0, 0, 0], [400, 400, 60], size=(20, 3)).astype(np.float32)
        r = o.sep_check(t0, traj)
        first = -1
        count = 0
        for k in range(len(traj)):
            for pt0, xyz in plans:
                j = t0 + k - pt0
                if 0 <= j < len(xyz):
                    hd = cdist(traj[k:k + 1, :2].astype(np.float64), xyz[j:j + 1, :2].astype(np.float64))[0, 0]
                    vd = abs(float(traj[k, 2]) - float(xyz[j, 2]))
                    if hd < 150.0 and vd < 30.0:
                        count += 1
                        first = k if first < 0 else first
        assert r["conflicts"] == count and r["first_conflict"] == first


# ---------------------------------------------------------------- invariants and FCFS


def _c1_small(n_plans=60, n_req=6, seed=21):
    sc = S.c1_plain_small(seed)
    sc.plans = sc.plans[:n_plans]
    sc.requests = sc.requests[:n_req]
    return sc


def test_mirror_symmetry():
    """Reflecting the whole scenario across y = 0 mirrors every trajectory exactly and
    swaps left and right turns."""
    sc = _c1_small()
    box = (0.0, -5000.0, 0.0, 10000.0, 5000.0, 500.0)
    shift = np.array([0.0, -5000.0, 0.0], dtype=np.float32)
    mirror = [ACT15.index((-d, c)) for d, c in ACT15]
    o1 = Oracle(box, 1.0, 0.99, ACT15, (150.0, 30.0))
    o2 = Oracle(box, 1.0, 0.99, ACT15, (150.0, 30.0))
    for pl in sc.plans:
        p = pl.xyz + shift
        o1.add_plan(pl.t0, p)
        o2.add_plan(pl.t0, p * np.array([1, -1, 1], dtype=np.float32))
    for r in sc.requests:
        a = dict(ox=r["ox"], oy=r["oy"] - 5000.0, oz=r["oz"], gx=r["gx"], gy=r["gy"] - 5000.0, gz=r["gz"],
                 speed=r["speed"], depart=r["depart"], horizon=r["horizon"])
        b = dict(a, oy=-a["oy"], gy=-a["gy"])
        d1, d2 = o1.rollout(a), o2.rollout(b)
        n = min(d1["n_points"], d2["n_points"])
        same = np.nonzero(d1["actions"][: n - 1] != np.array(mirror)[d2["actions"][: n - 1]])[0]
        # identical until the first exact tie broken by index order (none expected here)
        assert same.size == 0
        assert d1["n_points"] == d2["n_points"] and d1["verdict"] == d2["verdict"]
        np.testing.assert_array_equal(d1["xyz"], d2["xyz"] * np.array([1, -1, 1], dtype=np.float32))


def test_plan_order_permutation_invariance():
    sc = _c1_small(n_req=4)
    perm = np.random.default_rng(1).permutation(len(sc.plans))
    for combine in (0, 1):
        o1 = Oracle.from_scenario(sc, combine=combine)
        o2 = Oracle(sc.box, sc.dt, sc.gamma, sc.actions, sc.sep, combine=combine)
        for i in perm:
            o2.add_plan(sc.plans[i].t0, sc.plans[i].xyz)
        for r in sc.requests:
            d1, d2 = o1.rollout(r, trace=True), o2.rollout(r, trace=True)
            if combine == 0:
                np.testing.assert_array_equal(d1["q"], d2["q"])
                np.testing.assert_array_equal(d1["xyz"], d2["xyz"])
            else:
                np.testing.assert_allclose(d1["q"][:20], d2["q"][:20], rtol=1e-12)


def test_locality_far_plan_changes_nothing():
    sc = _c1_small(n_req=5)
    o1 = Oracle.from_scenario(sc)
    o2 = Oracle.from_scenario(sc)
    # a plan far outside every well of every successor (other corner, far above the box)
    o2.add_plan(0, np.tile(np.array([[-50000.0, -50000.0, 9000.0]], dtype=np.float32), (3000, 1)))
    for r in sc.requests:
        d1, d2 = o1.rollout(r, trace=True), o2.rollout(r, trace=True)
        np.testing.assert_array_equal(d1["q"], d2["q"])
        np.testing.assert_array_equal(d1["xyz"], d2["xyz"])


def test_time_shift_invariance():
    sc = _c1_small(n_req=4)
    o1 = Oracle.from_scenario(sc)
    o2 = Oracle(sc.box, sc.dt, sc.gamma, sc.actions, sc.sep)
    for pl in sc.plans:
        o2.add_plan(pl.t0 + 1000, pl.xyz)
    for r in sc.requests:
        r2 = {k: r[k] for k in r.dtype.names}
        r2["depart"] = int(r["depart"]) + 1000
        d1, d2 = o1.rollout(r, trace=True), o2.rollout(r2, trace=True)
        np.testing.assert_array_equal(d1["q"], d2["q"])


def test_fcfs_admitted_plan_blocks_identical_request():
    """Sec. V: an accepted plan is stored and used by every later request. The same
    request submitted twice starts inside the first one's plan: conflict at the origin."""
    o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    r = req(1000, 1000, 200, 8000, 7000, 250, speed=30.0, depart=5, horizon=800)
    d1 = o.schedule(r)
    assert d1["verdict"] == ADMITTED and d1["plan_id"] == 1 and o.n_plans == 1
    d2 = o.schedule(r)
    assert d2["verdict"] == REJ_CONFLICT and d2["first_conflict"] == 0 and o.n_plans == 1
    # the same request an hour later sees an empty sky again
    d3 = o.schedule(dict(r, depart=3605))
    assert d3["verdict"] == ADMITTED
    np.testing.assert_array_equal(d3["xyz"], d1["xyz"])


def test_known_plan_on_the_path_is_avoided():
    """A plan hovering on the straight path when the request would pass: the greedy value
    keeps the request out of its wells' core, so the admitted path keeps separation."""
    o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    o.add_plan(0, np.tile(np.array([[5000.0, 5000.0, 200.0]], dtype=np.float32), (1000, 1)))
    d = o.schedule(req(1000, 5000, 200, 9000, 5000, 200, speed=30.0, depart=0, horizon=800))
    assert d["verdict"] == ADMITTED
    assert d["min_sep_h"] > 150.0 or d["min_sep_v"] >= 30.0
    assert np.any(d["actions"] != ACT15.index((0.0, 0.0)))


def test_horizon_and_no_action_and_capture_at_origin():
    o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    d = o.schedule(req(1000, 1000, 200, 9000, 9000, 200, speed=30.0, horizon=10))
    assert d["verdict"] == REJ_HORIZON and d["n_points"] == 11
    # the goal lies outside the box behind the west wall: every successor leaves the box
    d = o.schedule(req(0.0, 5000, 200, -3000, 5000, 200, speed=30.0, horizon=10))
    assert d["verdict"] == REJ_NO_ACTION and d["n_points"] == 1
    d = o.schedule(req(1000, 1000, 200, 1010, 1020, 205, speed=30.0, horizon=10))
    assert d["verdict"] == ADMITTED and d["n_points"] == 1


def test_c1_fcfs_runs_and_is_deterministic():
    sc = S.c1_plain_small()
    o1 = Oracle.from_scenario(sc)
    o2 = Oracle.from_scenario(sc)
    v1 = [o1.schedule(r) for r in sc.requests[:12]]
    v2 = [o2.schedule(r) for r in sc.requests[:12]]
    for a, b in zip(v1, v2):
        assert a["verdict"] == b["verdict"]
        np.testing.assert_array_equal(a["xyz"], b["xyz"])
    assert sum(v["verdict"] == ADMITTED for v in v1) >= 8


def test_exact_ties_go_to_the_lowest_action_index():
    """Alg. 9 takes the argmax; on exact ties the first (lowest-index) action wins.

    Bearing +x makes the +-15 / +-30 deg successors exact mirror images about the track,
    and a static well dead ahead at the aircraft's altitude makes climb -2 and +2 mirror
    images too: the best value is shared by four actions, the lowest being (-30, -2)."""
    sw = np.array([[1035.0, 5000.0, 200.0, 40.0, 1000.0, 0.99]])
    o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0), static_wells=sw)
    q = o.q_values([1000.0, 5000.0, 200.0], 0, 0, 30.0, origin=[1000.0, 5000.0], goal=[9000.0, 5000.0, 200.0])
    best = np.flatnonzero(q["Q"] == q["Q"].max())
    assert list(best) == [ACT15.index(a) for a in ((-30.0, -2.0), (-30.0, 2.0), (30.0, -2.0), (30.0, 2.0))]
    d = o.rollout(req(1000.0, 5000.0, 200.0, 9000.0, 5000.0, 200.0, speed=30.0, horizon=1))
    assert d["actions"][0] == 0


def test_threaded_oracle_gives_the_same_results():
    """The multi-core oracle (a step's actions valued on several threads) computes every
    value as the single-threaded one does: identical trajectories, values and verdicts."""
    import oracle as O
    from paper_2008_03518_gb300 import scenarios as S

    sc = S.c1_plain_small()
    out = []
    try:
        for n in (1, 4):
            O.set_threads(n)
            o = O.Oracle.from_scenario(sc)
            out.append([o.schedule(r) for r in sc.requests[:6]])
    finally:
        O.set_threads(1)
    for a, b in zip(*out):
        assert a["verdict"] == b["verdict"]
        np.testing.assert_array_equal(a["xyz"], b["xyz"])
