"""The serving loop (fmdp_serve): continuous batching over a Poisson arrival trace.

Requests that arrive while others are on the device join the unresolved set as room and
plan slots allow, and are planned in the same speculative waves. Each result must be the
same as when the requests are scheduled one at a time in arrival order (alone), bit for
bit, whatever the mix, the expiry clock and the memory-based admission did.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import ADMITTED  # noqa: E402
from paper_2008_03518_gb300 import scenarios as S  # noqa: E402
from paper_2008_03518_gb300.fmdp import Scheduler  # noqa: E402

from parity_util import fcfs_parity, follow_and_check, oracle_for  # noqa: E402
from test_gpu_batch import same_results, same_tables, table_of  # noqa: E402


def poisson(n, rate, seed):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def test_served_results_equal_one_at_a_time():
    sc = S.crowded_batch(seed=111, n_requests=60)
    arr = poisson(len(sc.requests), 2000.0, 1)
    with Scheduler.from_scenario(sc) as s:
        alone = s.schedule_many(sc.requests)
        t_alone = table_of(s)
    with Scheduler.from_scenario(sc, batch_size=32) as s:
        mixed, lat, rep = s.serve(sc.requests, arr)
        t_mixed = table_of(s)
    same_results(alone, mixed)
    same_tables(t_alone, t_mixed)
    assert rep["admitted"] == sum(r["verdict"] == ADMITTED for r in alone)
    assert rep["admitted"] + rep["rejected"] == len(sc.requests)
    assert (lat > 0).all() and rep["latency_p99_ms"] >= rep["latency_p50_ms"] > 0
    assert rep["max_in_flight_seen"] > 1  # requests were planned side by side
    assert rep["pipelined"] == 1 and rep["waves"] == 0 and rep["rollouts"] >= len(sc.requests)
    assert 0.0 < rep["rollout_occupancy"] <= 1.0
    assert rep["throughput_rps"] > 0


def test_wave_serving_equals_one_at_a_time():
    """The same trace served by speculative waves (batch_mode 1)."""
    sc = S.crowded_batch(seed=111, n_requests=60)
    arr = poisson(len(sc.requests), 2000.0, 1)
    with Scheduler.from_scenario(sc) as s:
        alone = s.schedule_many(sc.requests)
    with Scheduler.from_scenario(sc, batch_size=32, batch_mode=1) as s:
        mixed, lat, rep = s.serve(sc.requests, arr)
    same_results(alone, mixed)
    assert rep["pipelined"] == 0 and rep["waves"] >= 1


def test_served_results_match_the_oracle():
    """Every served request re-derived by the FP64 oracle, in arrival order, from the table
    the GPU had when it planned it (the known plans plus every request admitted before it):
    trajectories bit for bit, action sequences equal except at the oracle's own near-ties,
    verdicts and first-conflict steps identical, minimum separations within 1e-5."""
    sc = S.crowded_batch(seed=112, n_requests=48)
    arr = poisson(len(sc.requests), 2000.0, 3)
    with Scheduler.from_scenario(sc, batch_size=32) as s:
        served, lat, rep = s.serve(sc.requests, arr)
    verdicts, _, _ = fcfs_parity(None, oracle_for(sc), sc.requests, gpu_results=served)
    assert sum(v == ADMITTED for v in verdicts) == rep["admitted"] > 0
    assert rep["admitted"] < len(sc.requests)  # the mix also rejects
    assert rep["max_in_flight_seen"] > 1


def _staggered(sc, gap):
    """Requests departing one after another, `gap` steps apart, from step 200 on."""
    r = sc.requests.copy()
    r["depart"] = 200 + gap * np.arange(len(r))
    r["horizon"] = np.minimum(r["horizon"], 600)
    return r


def test_serving_expires_finished_plans_without_changing_results():
    sc = S.c1_plain_small()
    reqs = _staggered(sc, 12)[:40]
    arr = np.linspace(0.0, 0.4, len(reqs))
    with Scheduler.from_scenario(sc) as s:
        alone = s.schedule_many(reqs)
    with Scheduler.from_scenario(sc) as s:
        # 2000 simulated seconds per wall second: the clock passes the known plans' ends
        mixed, lat, rep = s.serve(reqs, arr, time_scale=2000.0, expire_quantum=30)
        remaining = len(s.query_plans(-(1 << 40), 1 << 40))
    same_results(alone, mixed)
    assert rep["expiries"] > 0 and rep["plans_expired"] > 0
    assert remaining == len(sc.plans) + rep["admitted"] - rep["plans_expired"]
    assert rep["final_t_base"] <= int(reqs["depart"].max())


def test_served_with_expiry_matches_the_oracle():
    """Expiry removes only plans that ended before every departure still to plan, so the
    oracle, which keeps every plan, derives the same results for every served request."""
    sc = S.c1_plain_small()
    reqs = _staggered(sc, 12)[:40]
    arr = np.linspace(0.0, 0.4, len(reqs))
    with Scheduler.from_scenario(sc) as s:
        served, lat, rep = s.serve(reqs, arr, time_scale=2000.0, expire_quantum=30)
    assert rep["plans_expired"] > 0
    verdicts, _, _ = fcfs_parity(None, oracle_for(sc), reqs, gpu_results=served)
    assert sum(v == ADMITTED for v in verdicts) == rep["admitted"]


def test_memory_based_admission_defers_and_keeps_results():
    sc = S.c1_plain_small()
    reqs = _staggered(sc, 15)[:30]
    arr = np.zeros(len(reqs))  # all arrive at once
    with Scheduler.from_scenario(sc) as s:
        alone = s.schedule_many(reqs)
    with Scheduler.from_scenario(sc) as s:
        # room for only four more plans than the known ones: requests wait for expiries
        mixed, lat, rep = s.serve(reqs, arr, time_scale=5000.0, expire_quantum=20,
                                  max_active_plans=len(sc.plans) + 4)
    same_results(alone, mixed)
    # arrivals waited for room; the unresolved set grows only as expiries free plans
    assert rep["deferred_for_memory"] > 0 and rep["max_in_flight_seen"] < len(reqs)
    assert rep["expiries"] > 0


def test_full_table_with_nothing_to_expire_is_an_error():
    sc = S.c1_plain_small()
    reqs = _staggered(sc, 5)[:10]
    from paper_2008_03518_gb300.fmdp import FmdpError

    with Scheduler.from_scenario(sc, add_plans=False) as s:
        # eight plans that outlive every request's departure fill the allowed table
        far = np.array([[9900.0, 9900.0, 480.0]], dtype=np.float32)
        for k in range(8):
            s.add_plan(0, np.repeat(far + np.float32(10.0 * k), 1500, axis=0))
        with pytest.raises(FmdpError) as e:
            s.serve(reqs, np.zeros(len(reqs)), time_scale=1.0, max_active_plans=8)
        assert "full" in str(e.value)


def test_c4_shape_100k_plans_sampled_against_the_oracle():
    """Serving at the C4 shape: C2's 30 km airspace and terrain, 100k known plans in the
    sliding-window table (memory-based admission at 100k active plans, expiry from the
    simulated clock), Poisson arrivals. Sampled served requests are re-derived by the FP64
    oracle from the table the GPU had when it planned them (the known plans and every
    request admitted before them), on all host cores."""
    import os

    import oracle as O

    sc = S.c4_serving()
    sim0 = sc.meta["sim_start"]
    arr = S.poisson_arrivals(77, 1000.0, 0.5)
    reqs = S.serving_requests(sc, arr, 78, time_scale=60.0, sim_start=sim0)
    with Scheduler.from_scenario(sc) as s:
        served, lat, rep = s.serve(reqs, arr, time_scale=60.0, max_active_plans=sc.meta["max_active_plans"],
                                   sim_start_step=sim0)
    assert rep["pipelined"] == 1 and rep["expiries"] >= 1 and rep["plans_expired"] > 0
    assert rep["admitted"] > 0 and rep["admitted"] + rep["rejected"] == len(reqs)
    adm = [i for i, r in enumerate(served) if r["verdict"] == ADMITTED]
    rej = [i for i, r in enumerate(served) if r["verdict"] != ADMITTED]
    picks = sorted({adm[0], adm[-1], rej[len(rej) // 2]})
    O.set_threads(os.cpu_count() or 1)
    try:
        o = oracle_for(sc)
        done = 0
        for k in picks:
            for i in range(done, k):  # the oracle's table as the GPU had it before request k
                if served[i]["verdict"] == ADMITTED:
                    o.add_plan(int(reqs[i]["depart"]), served[i]["xyz"])
            done = k
            v, _ = follow_and_check(o, reqs[k], served[k])
            assert v == served[k]["verdict"], k
    finally:
        O.set_threads(1)
