"""Departure-time candidates on the GPU (fmdp_schedule_departures): the variants of a
request departing later are planned together and the first admissible one is admitted.

- against the oracle on the hover scenario, whose outcome is pinned in closed form;
- against trying the variants one at a time with fmdp_schedule (the definition: rejected
  variants change nothing), bit for bit, on C1 traffic;
- window and argument errors leave the table unchanged;
- the batched call (fmdp_schedule_departures_batch: the variants of many requests through
  speculative batches) equals the one-request-at-a-time call bit for bit, verdicts of every
  variant and the table included, with re-plans exercised.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import ADMITTED, Oracle  # noqa: E402
from paper_2008_03518_gb300 import scenarios as S  # noqa: E402
from paper_2008_03518_gb300.fmdp import FmdpError, Scheduler  # noqa: E402
from tests.parity_util import follow_and_check  # noqa: E402

from test_gpu_batch import same_results, same_tables, table_of  # noqa: E402

ACT15 = S.action_grid((-2.0, 0.0, 2.0))
BOX = (0.0, 0.0, 0.0, 10000.0, 10000.0, 500.0)
GOAL = (5000.0, 5000.0, 200.0)
HOVER = np.repeat(np.array([GOAL], dtype=np.float32), 301, axis=0)  # steps 0 .. 300


def request(depart=0, rid=7):
    return dict(id=rid, ox=2000.0, oy=5000.0, oz=200.0, gx=GOAL[0], gy=GOAL[1], gz=GOAL[2], speed=30.0,
                depart=depart, horizon=105)


def hover_pair():
    o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    o.add_plan(0, HOVER)
    s = Scheduler(BOX, 1.0, 0.99, ACT15, (150.0, 30.0), n_slices_window=2048, max_slots=64)
    s.add_plan(0, HOVER)
    return o, s


def variant(r, delay):
    v = dict(r) if isinstance(r, dict) else {k: r[k] for k in r.dtype.names}
    v["depart"] = int(v["depart"]) + int(delay)
    return v


def test_hover_scenario_matches_the_oracle():
    o, s = hover_pair()
    delays = [0, 20, 60, 400, 500]
    with s:
        res, chosen, verd = s.schedule_departures([request()], delays)
        n_plans = len(s.query_plans(-(1 << 40), 1 << 40))
    d, tried = o.schedule_departures(request(), delays)
    assert chosen[0] == d == 3
    assert list(verd[0][:4]) == [t["verdict"] for t in tried]
    assert verd[0][4] == ADMITTED  # the later variant is admissible too, but not taken
    g = res[0]
    assert g["verdict"] == ADMITTED and g["plan_id"] != 0 and n_plans == 2
    v, od = follow_and_check(Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0)), variant(request(), 400), g)
    assert v == ADMITTED
    np.testing.assert_array_equal(g["xyz"], tried[3]["xyz"])


def test_no_admissible_variant_returns_the_first_and_admits_nothing():
    o, s = hover_pair()
    with s:
        res, chosen, verd = s.schedule_departures([request()], [0, 10, 30])
        assert len(s.query_plans(-(1 << 40), 1 << 40)) == 1
        alone = s.schedule(request())
    assert chosen[0] == -1 and all(v != ADMITTED for v in verd[0])
    assert res[0]["verdict"] == verd[0][0] == alone["verdict"] and res[0]["plan_id"] == 0
    np.testing.assert_array_equal(res[0]["xyz"], alone["xyz"])


@pytest.mark.parametrize("full_scan", [False, True])
def test_equals_trying_the_variants_one_at_a_time(full_scan):
    sc = S.crowded_batch(seed=131, n_requests=16)
    delays = [0, 25, 50, 100, 200]
    with Scheduler.from_scenario(sc, full_scan=full_scan) as s:
        res, chosen, verd = s.schedule_departures(sc.requests, delays)
        t_cand = table_of(s)
    want, want_chosen, want_verd = [], [], []
    with Scheduler.from_scenario(sc, full_scan=full_scan) as s:
        for r in sc.requests:
            vs, pick, first = [], -1, None
            for k, dl in enumerate(delays):
                g = s.schedule(variant(r, dl))
                vs.append(g["verdict"])
                first = g if first is None else first
                if g["verdict"] == ADMITTED:
                    pick = k
                    want.append(g)
                    break
            if pick < 0:
                want.append(first)
            want_chosen.append(pick)
            want_verd.append(vs)
        t_seq = table_of(s)
    assert list(chosen) == want_chosen
    assert 0 < sum(c >= 0 for c in chosen) and any(c > 0 for c in chosen)  # delays mattered
    for i, vs in enumerate(want_verd):
        assert list(verd[i][:len(vs)]) == vs
    same_results(want, res)
    same_tables(t_seq, t_cand)


def test_window_and_argument_errors_leave_the_table_unchanged():
    o, s = hover_pair()
    with s:
        with pytest.raises(FmdpError) as e:
            s.schedule_departures([request()], [0, 5000])  # a variant beyond the window
        assert e.value.status == -6
        with pytest.raises(FmdpError):
            s.schedule_departures([request()], [])
        assert len(s.query_plans(-(1 << 40), 1 << 40)) == 1


@pytest.mark.parametrize("full_scan,batch_size", [(False, 0), (False, 10), (True, 0)])
def test_batched_equals_one_request_at_a_time(full_scan, batch_size):
    """batch_size 0: every request's variants in one batch (24 requests x 5 variants);
    10: two requests per batch."""
    sc = S.crowded_batch(seed=131, n_requests=24)
    delays = [0, 25, 50, 100, 200]
    with Scheduler.from_scenario(sc, full_scan=full_scan) as s:
        res, chosen, verd = s.schedule_departures(sc.requests, delays)
        t_seq = table_of(s)
    with Scheduler.from_scenario(sc, full_scan=full_scan, batch_size=batch_size) as s:
        bres, bchosen, bverd = s.schedule_departures(sc.requests, delays, batched=True)
        st = s.stats()
        t_bat = table_of(s)
    assert list(bchosen) == list(chosen) and any(c > 0 for c in chosen)
    np.testing.assert_array_equal(bverd, verd)
    same_results(res, bres)
    same_tables(t_seq, t_bat)
    assert st["batch_rollouts"] == len(sc.requests) * len(delays) + st["batch_replans"]
    if batch_size == 0:
        assert st["batch_replans"] > 0 and st["batch_waves"] > 1


def test_batched_hover_scenario_matches_the_oracle():
    o, s = hover_pair()
    delays = [0, 20, 60, 400, 500]
    with s:
        res, chosen, verd = s.schedule_departures([request(), request(depart=3, rid=8)], delays, batched=True)
    d, tried = o.schedule_departures(request(), delays)
    assert chosen[0] == d == 3
    assert list(verd[0][:4]) == [t["verdict"] for t in tried]
    np.testing.assert_array_equal(res[0]["xyz"], tried[3]["xyz"])


def test_batched_window_errors_leave_the_table_unchanged():
    o, s = hover_pair()
    with s:
        with pytest.raises(FmdpError) as e:
            s.schedule_departures([request(), request()], [0, 5000], batched=True)
        assert e.value.status == -6
        assert len(s.query_plans(-(1 << 40), 1 << 40)) == 1
