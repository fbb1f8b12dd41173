"""GPU parity: the CUDA scheduler (through the C ABI) against the FP64 oracle on the same
seeded inputs. Trajectories, verdicts and conflict indices must be bit-identical; action
values within 1e-5 of their term scale; actions identical except at recorded near-ties.
"""
import numpy as np
import pytest

from oracle import ADMITTED, REJ_CONFLICT, REJ_HORIZON, REJ_NO_ACTION, Oracle
from paper_2008_03518_gb300 import scenarios as S
from tests.parity_util import check_q, fcfs_parity, follow_and_check

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2008_03518_gb300.fmdp import FmdpError, Scheduler  # noqa: E402

ACT15 = S.action_grid((-2.0, 0.0, 2.0))
ACT25 = S.action_grid((-4.0, -2.0, 0.0, 2.0, 4.0))
BOX = (0.0, 0.0, 0.0, 10000.0, 10000.0, 500.0)


def req(ox, oy, oz, gx, gy, gz, speed=30.0, depart=0, horizon=600, rid=1):
    return dict(req_id=rid, ox=ox, oy=oy, oz=oz, gx=gx, gy=gy, gz=gz, speed=speed, depart=depart, horizon=horizon)


@pytest.fixture(scope="module")
def c1():
    return S.c1_plain_small()


def test_plan_table_roundtrip_and_query(c1):
    with Scheduler.from_scenario(c1, add_plans=False) as s:
        ids = s.add_plans([(p.t0, p.xyz) for p in c1.plans])
        assert len(set(ids.tolist())) == len(ids)
        for pid, p in zip(ids[::7], c1.plans[::7]):
            t0, xyz = s.get_plan(pid)
            assert t0 == p.t0
            np.testing.assert_array_equal(xyz, p.xyz)
        for a, b in ((0, 50), (300, 301), (0, 10 ** 6), (5000, 6000), (599, 600)):
            want = {int(ids[i]) for i, p in enumerate(c1.plans) if p.t0 < b and p.t0 + len(p.xyz) > a}
            assert set(int(x) for x in s.query_plans(a, b)) == want


def test_sep_check_parity_including_threshold_pairs():
    rng = np.random.default_rng(42)
    for trial in range(6):
        box = BOX
        s = Scheduler(box, 1.0, 0.99, ACT15, (150.0, 30.0), n_slices_window=256, max_slots=300 + trial * 37)
        o = Oracle(box, 1.0, 0.99, ACT15, (150.0, 30.0))
        base = rng.uniform([2000, 2000, 100], [3000, 3000, 300], size=(40, 3)).astype(np.float32)
        plans = []
        for j in range(250 + trial * 37):
            t0 = int(rng.integers(0, 20))
            xyz = (base[rng.integers(0, 40)] + rng.uniform(-400, 400, size=(int(rng.integers(5, 60)), 3))).astype(np.float32)
            plans.append((t0, xyz))
        s.add_plans(plans)
        for t0, xyz in plans:
            o.add_plan(t0, xyz)
        for q in range(8):
            t0 = int(rng.integers(0, 20))
            traj = (base[rng.integers(0, 40)] + rng.uniform(-400, 400, size=(50, 3))).astype(np.float32)
            # plant pairs exactly at, just inside and just outside the minima (1e-3 m is a few
            # fp32 ulps at these coordinates, 3e-5 m below one: the sum rounds to the nearest
            # representable sample, so those pairs sit within an ulp or two of the minima)
            for k in range(0, 50, 5):
                j = int(rng.integers(0, len(plans)))
                pt0, pxyz = plans[j]
                idx = t0 + k - pt0
                if 0 <= idx < len(pxyz):
                    off = rng.choice([150.0, 149.999, 150.001, 149.99997, 150.00003, 0.0])
                    dz = rng.choice([30.0, 29.999, 30.001, 29.99997, 30.00003, 0.0])
                    ang = rng.uniform(0, 2 * np.pi)
                    traj[k] = pxyz[idx] + np.array([off * np.cos(ang), off * np.sin(ang), dz], dtype=np.float32)
            g = s.sep_check(t0, traj)
            r = o.sep_check(t0, traj)
            assert g["conflicts"] == r["conflicts"]
            assert g["first_conflict_step"] == r["first_conflict"]
            for k in ("min_sep_h", "min_sep_v"):
                if np.isfinite(r[k]):
                    assert g[k] == pytest.approx(r[k], rel=1e-5, abs=1e-5)
                else:
                    assert not np.isfinite(g[k])
        s.close()


def test_c1_lockstep_q_and_fcfs(c1):
    """Config 1 in full: 200 known plans, 50 FCFS requests, 15 actions."""
    with Scheduler.from_scenario(c1) as s:
        o = Oracle.from_scenario(c1)
        verdicts, followed, steps = fcfs_parity(s, o, c1.requests, trace_q=True)
    assert sum(v == ADMITTED for v in verdicts) >= 30
    # the GPU may take the other action of an exact or near tie (gap < 1e-4 of the scale)
    assert followed <= max(5, steps // 1000), (followed, steps)


@pytest.mark.parametrize("cs", [1, 2, 4, 8, 16])
def test_cluster_split_is_bit_identical(c1, cs):
    """Full-scan rollouts: the slot range split over clusters of 1 to 16 CTAs."""
    sc = c1
    with Scheduler.from_scenario(sc, cluster_size=1, full_scan=True) as ref, \
            Scheduler.from_scenario(sc, cluster_size=cs, full_scan=True) as s:
        for r in sc.requests[:6]:
            a, b = ref.rollout_trace(r), s.rollout_trace(r)
            np.testing.assert_array_equal(a["xyz"], b["xyz"])
            np.testing.assert_array_equal(a["q"], b["q"])


def test_sum_mode_parity(c1):
    sc = S.c1_plain_small()
    sc.requests = sc.requests[:15]
    with Scheduler.from_scenario(sc, combine=1) as s:
        o = Oracle.from_scenario(sc, combine=1)
        fcfs_parity(s, o, sc.requests, trace_q=True)


def _terrain_scenario(seed=7, n_plans=400, n_req=12, low=True):
    hm = S.fractal_heightmap(seed, n=129, top=300.0)
    rng = np.random.default_rng(seed)
    box = (0.0, 0.0, 0.0, 12000.0, 12000.0, 1000.0)
    plans = S.multileg_plans(rng, box, n_plans, hm, legs=(2, 4), leg_len=(1500.0, 5000.0), tlo=0, thi=600)
    reqs = S.make_requests(rng, box, n_req, hm=hm, zspan=(5.0, 120.0) if low else (60.0, 400.0), tlo=0, thi=600,
                           horizon=1500)
    sw = np.array([[6000.0, 6000.0, 300.0, 800.0, 1000.0, 0.99], [3000.0, 9000.0, 200.0, 400.0, 500.0, 0.98],
                   [9000.0, 2500.0, 500.0, 1200.0, 1000.0, 0.99]])
    return S.Scenario("terrain_small", box, 1.0, 0.99, ACT25, (150.0, 30.0), plans, reqs, heightmap=hm,
                      clearance=60.0, static_wells=sw, n_slices_window=4096, max_slots=n_plans + n_req + 64)


def test_terrain_static_wells_parity():
    sc = _terrain_scenario()
    with Scheduler.from_scenario(sc) as s:
        o = Oracle.from_scenario(sc)
        fcfs_parity(s, o, sc.requests, trace_q=True)


def test_c2_scale_subset():
    """Config 2's airspace at full scale (3000 multi-leg plans, terrain, 25 actions); the
    first 12 FCFS requests checked in lock step."""
    sc = S.c2_plain_scale()
    with Scheduler.from_scenario(sc) as s:
        o = Oracle.from_scenario(sc)
        fcfs_parity(s, o, sc.requests[:12], trace_q=True)


def test_schedule_many_and_staged_equal_sequential(c1):
    sc = c1
    reqs = sc.requests[:20]
    with Scheduler.from_scenario(sc) as a, Scheduler.from_scenario(sc) as b, Scheduler.from_scenario(sc) as c:
        seq = [a.schedule(r) for r in reqs]
        many = b.schedule_many(reqs)
        c.stage(reqs)
        c.schedule_staged()
        staged = c.fetch_staged()
        for x, y, z in zip(seq, many, staged):
            assert x["verdict"] == y["verdict"] == z["verdict"]
            np.testing.assert_array_equal(x["xyz"], y["xyz"])
            np.testing.assert_array_equal(x["xyz"], z["xyz"])
            assert x["plan_id"] == y["plan_id"]
        assert set(a.query_plans(0, 10 ** 6)) == set(b.query_plans(0, 10 ** 6)) == set(c.query_plans(0, 10 ** 6))


def test_edge_cases():
    with Scheduler(BOX, 1.0, 0.99, ACT15, (150.0, 30.0), n_slices_window=1024, max_slots=40) as s:
        o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
        # empty table: straight flight
        r = req(1000, 1000, 200, 6000, 4000, 200, horizon=400)
        g = s.schedule(r)
        v, _ = follow_and_check(o, r, g)
        assert g["verdict"] == v == ADMITTED and np.all(g["actions"] == ACT15.index((0.0, 0.0)))
        o.add_plan(0, g["xyz"])
        # horizon exhausted, zero horizon, capture at the origin, dead end
        for rr, want in ((req(1000, 9000, 200, 9000, 1000, 200, horizon=5), REJ_HORIZON),
                         (req(1000, 9000, 200, 9000, 1000, 200, horizon=0), REJ_HORIZON),
                         (req(3000, 3000, 100, 3010, 3005, 104), ADMITTED),
                         (req(0.0, 5000, 200, -3000, 5000, 200, horizon=20), REJ_NO_ACTION)):
            g = s.schedule(rr)
            v, d = follow_and_check(o, rr, g)
            assert g["verdict"] == v == want
            if v == ADMITTED:
                o.add_plan(rr["depart"], d["xyz"])
        # the identical request again conflicts at its origin
        g = s.schedule(r)
        assert g["verdict"] == REJ_CONFLICT and g["first_conflict_step"] == 0
        # window: a request beyond the table's time window is refused, not planned
        with pytest.raises(FmdpError) as e:
            s.schedule(req(1000, 1000, 200, 6000, 4000, 200, depart=1000, horizon=100))
        assert e.value.status == -6
        # table full
        n_free = 40 - len(s.query_plans(0, 10 ** 6))
        s.add_plans([(0, np.array([[50.0 * i, 50.0, 450.0]], dtype=np.float32)) for i in range(n_free)])
        with pytest.raises(FmdpError) as e:
            s.add_plan(0, np.zeros((1, 3), dtype=np.float32))
        assert e.value.status == -5
        # non-finite points are rejected
        with pytest.raises(FmdpError):
            s.add_plan(0, np.array([[np.nan, 0, 0]], dtype=np.float32))


def test_ragged_slot_counts_and_expiry():
    rng = np.random.default_rng(3)
    for n_plans in (1, 31, 33, 97):
        plans = S.straight_plans(rng, BOX, n_plans, 50.0, 450.0, 20.0, 40.0, 0, 100, 1.0)
        reqs = S.make_requests(rng, BOX, 4, tlo=0, thi=100, horizon=900)
        sc = S.Scenario("ragged", BOX, 1.0, 0.99, ACT15, (150.0, 30.0), plans, reqs, n_slices_window=2048,
                        max_slots=n_plans + 8)
        with Scheduler.from_scenario(sc) as s:
            fcfs_parity(s, Oracle.from_scenario(sc), reqs)
    # expiry frees slots and clears rows; a later plan can reuse the slot
    with Scheduler(BOX, 1.0, 0.99, ACT15, (150.0, 30.0), n_slices_window=64, max_slots=2) as s:
        a = s.add_plan(0, np.tile(np.array([[100, 100, 100]], dtype=np.float32), (10, 1)))
        b = s.add_plan(5, np.tile(np.array([[900, 900, 100]], dtype=np.float32), (50, 1)))
        s.expire(20)
        assert set(s.query_plans(0, 10 ** 6)) == {b}
        c = s.add_plan(30, np.tile(np.array([[500, 500, 100]], dtype=np.float32), (40, 1)))
        assert c not in (a, b)
        rep = s.sep_check(40, np.array([[500, 500, 100]], dtype=np.float32))
        assert rep["conflicts"] == 1
        rep = s.sep_check(10, np.array([[100, 100, 100]], dtype=np.float32))
        assert rep["conflicts"] == 0  # a's rows left with the window


def test_snapshot_restore(c1):
    with Scheduler.from_scenario(c1) as s:
        s.snapshot()
        first = s.schedule_many(c1.requests[:5])
        s.restore()
        again = s.schedule_many(c1.requests[:5])
        for x, y in zip(first, again):
            assert x["verdict"] == y["verdict"]
            np.testing.assert_array_equal(x["xyz"], y["xyz"])


def test_full_size_c2_sampled():
    """Config 2 at full size in the launch configuration the benchmark times (one FCFS
    sequence of 1000 requests enqueued without host round trips); sampled requests are
    re-derived by the oracle from the table state the GPU had when it planned them."""
    sc = S.c2_plain_scale()
    with Scheduler.from_scenario(sc) as s:
        res = s.schedule_many(sc.requests)
    admitted = [(int(sc.requests[i]["depart"]), r["xyz"]) for i, r in enumerate(res) if r["verdict"] == ADMITTED]
    assert len(admitted) > 100
    picks = [0, 1, 137, 402, 655, 999]
    o = Oracle.from_scenario(sc)
    done = 0
    for k in picks:
        for i in range(done, k):  # bring the oracle's table to the state before request k
            if res[i]["verdict"] == ADMITTED:
                o.add_plan(int(sc.requests[i]["depart"]), res[i]["xyz"])
        done = k
        v, _ = follow_and_check(o, sc.requests[k], res[k])
        assert v == res[k]["verdict"], k
