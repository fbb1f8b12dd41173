"""Batch co-simulation on the GPU (fmdp_schedule_cosim) against the oracle's restatement
(pinned in test_oracle_cosim.py): the requests of a batch step on one clock and see each
other's wells; the trajectories must equal the oracle's bit for bit (the oracle takes the
GPU's action at recorded near-ties), and so must the verdicts of the array-order admission.
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

ACT15 = S.action_grid((-2.0, 0.0, 2.0))
BOX = (0.0, 0.0, 0.0, 10000.0, 10000.0, 500.0)


def cosim_parity(s, o, reqs):
    got = s.schedule_cosim(reqs)
    want = o.schedule_cosim(reqs, follow=[g["actions"] for g in got])
    for i, (g, w) in enumerate(zip(got, want)):
        assert w["mismatch_step"] == -1, f"request {i}: GPU action not a near-tie at step {w['mismatch_step']}"
        assert g["n_points"] == w["n_points"], i
        np.testing.assert_array_equal(g["xyz"], w["xyz"], err_msg=f"request {i}")
        assert g["verdict"] == w["verdict"], (i, g["verdict"], w["verdict"])
        if w["captured"]:
            assert g["first_conflict_step"] == w["first_conflict"]
    return got, want


def test_head_on_pair_matches_the_oracle_and_keeps_separation():
    reqs = [dict(id=1, ox=2000.0, oy=5000.0, oz=200.0, gx=8000.0, gy=5000.0, gz=200.0, speed=30.0, depart=0,
                 horizon=400),
            dict(id=2, ox=8000.0, oy=5000.0, oz=200.0, gx=2000.0, gy=5000.0, gz=200.0, speed=30.0, depart=0,
                 horizon=400)]
    o = Oracle(BOX, 1.0, 0.99, ACT15, (150.0, 30.0))
    with Scheduler(BOX, 1.0, 0.99, ACT15, (150.0, 30.0), n_slices_window=2048, max_slots=64) as s:
        got, _ = cosim_parity(s, o, reqs)
    assert [g["verdict"] for g in got] == [ADMITTED, ADMITTED]


@pytest.mark.parametrize("W,combine", [(1, 0), (1, 1), (3, 0)])
def test_crowded_batch_matches_the_oracle(W, combine):
    sc = S.crowded_batch(seed=141, n_requests=24)
    o = Oracle.from_scenario(sc, lookahead_W=W, combine=combine)
    with Scheduler.from_scenario(sc, lookahead_W=W, combine=combine) as s:
        got, want = cosim_parity(s, o, sc.requests)
        n_plans = len(s.query_plans(-(1 << 40), 1 << 40))
    adm = sum(g["verdict"] == ADMITTED for g in got)
    assert adm > 0 and n_plans == len(sc.plans) + adm


def test_staggered_departures_and_terrain():
    sc = S.c2_plain_scale(n_plans=300, n_requests=10)
    reqs = sc.requests.copy()
    reqs["depart"] = 100 + 7 * np.arange(len(reqs))
    reqs["horizon"] = np.minimum(reqs["horizon"], 900)
    o = Oracle.from_scenario(sc)
    with Scheduler.from_scenario(sc) as s:
        cosim_parity(s, o, reqs)


def test_batch_too_large_for_one_launch_is_refused():
    sc = S.c1_plain_small()
    rng = np.random.default_rng(1)
    many = S.make_requests(rng, sc.box, 4000, tlo=0, thi=600, horizon=100)
    with Scheduler.from_scenario(sc, max_slots=8192) as s:
        with pytest.raises(FmdpError) as e:
            s.schedule_cosim(many)
        assert e.value.status == -1
        assert len(s.query_plans(-(1 << 40), 1 << 40)) == len(sc.plans)


def test_a_wait_that_runs_out_reports_a_timeout_and_the_context_survives():
    """Failure detection without a fault: a grid barrier that waits for an aircraft that is
    never launched expires (bounded wait), the call reports FMDP_ERR_TIMEOUT, and the same
    context then plans normally."""
    sc = S.crowded_batch(seed=141, n_requests=6)
    with Scheduler.from_scenario(sc) as s:
        assert s.selftest_wait_timeout() == -4
        got = s.schedule_cosim(sc.requests)
        assert all(g["n_points"] >= 1 for g in got)
        alone = s.schedule(sc.requests[0])
        assert alone["n_points"] >= 1
