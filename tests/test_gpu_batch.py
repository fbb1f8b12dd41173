"""Batched speculative FCFS (fmdp_schedule_batch) against sequential FCFS.

The batch path plans many requests at once against the table as it stands and replans
only those an earlier admission of the same batch may have changed. It runs in two modes:
pipelined (batch_mode 0, the default: one persistent rollout launch fed by the host, no
waves) and speculative waves (batch_mode 1); both are checked. Its results must be
identical, bit for bit, to planning the requests one after the other (fmdp_schedule_many,
itself checked against the FP64 oracle in test_gpu_parity.py), and the table it leaves
must hold the same plans. The crowded scenario makes the requests' paths cross so that
the replan path is exercised; a few cases also go straight to the oracle.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import ADMITTED  # noqa: E402
from paper_2008_03518_gb300 import scenarios as S  # noqa: E402
from paper_2008_03518_gb300.fmdp import FmdpError, Scheduler  # noqa: E402

from parity_util import fcfs_parity, oracle_for  # noqa: E402

KEYS = ("verdict", "n_points", "first_conflict_step", "first_terrain_step", "plan_id", "near_ties",
        "min_sep_h", "min_sep_v")


def same_results(a, b):
    assert len(a) == len(b)
    for i, (x, y) in enumerate(zip(a, b)):
        for k in KEYS:
            assert x[k] == y[k] or (np.isnan(x[k]) and np.isnan(y[k])), (i, k, x[k], y[k])
        np.testing.assert_array_equal(x["xyz"], y["xyz"], err_msg=f"request {i}")
        np.testing.assert_array_equal(x["actions"], y["actions"], err_msg=f"request {i}")


def table_of(s, t_end=1 << 40):
    ids = s.query_plans(-(1 << 40), t_end)
    out = {}
    for i in ids:
        try:
            out[int(i)] = s.get_plan(i)
        except FmdpError as e:  # a plan that started before the window's first step
            out[int(i)] = (e.status, np.zeros((0, 3), np.float32))
    return out


def same_tables(a, b):
    assert a.keys() == b.keys()
    for k in a:
        assert a[k][0] == b[k][0]
        np.testing.assert_array_equal(a[k][1], b[k][1])


def run_both(sc, reqs=None, **kw):
    reqs = sc.requests if reqs is None else reqs
    with Scheduler.from_scenario(sc, **kw) as s1:
        many = s1.schedule_many(reqs)
        t1 = table_of(s1)
    with Scheduler.from_scenario(sc, **kw) as s2:
        bat = s2.schedule_batch(reqs)
        t2 = table_of(s2)
        st = s2.stats()
    return many, bat, t1, t2, st


@pytest.mark.parametrize("batch_mode", [0, 1])
@pytest.mark.parametrize("batch_size", [0, 16])
def test_batch_equals_sequential_c1(batch_size, batch_mode):
    sc = S.c1_plain_small()
    many, bat, t1, t2, st = run_both(sc, batch_size=batch_size, batch_mode=batch_mode)
    same_results(many, bat)
    same_tables(t1, t2)
    assert sum(r["verdict"] == ADMITTED for r in bat) > 0
    assert st["batch_rollouts"] >= len(sc.requests)


@pytest.mark.parametrize("cs", [0, 2, 4])
def test_crowded_batch_replans_and_matches(cs):
    sc = S.crowded_batch()
    many, bat, t1, t2, st = run_both(sc, cluster_size=cs, batch_mode=1)
    same_results(many, bat)
    same_tables(t1, t2)
    # the paths cross: some requests were planned again, and the walk took several waves
    assert st["batch_replans"] > 0 and st["batch_waves"] > 1
    assert sum(r["replanned"] for r in bat) == st["batch_replans"]
    assert st["batch_rollouts"] == len(sc.requests) + st["batch_replans"]


@pytest.mark.parametrize("batch_size", [0, 4])
def test_pipelined_crowded_batch_replans_and_matches(batch_size):
    """Pipelined mode (no waves): the crossing paths force re-plans, every re-plan is
    counted once, and the results and the table equal sequential FCFS."""
    sc = S.crowded_batch()
    many, bat, t1, t2, st = run_both(sc, batch_size=batch_size)
    same_results(many, bat)
    same_tables(t1, t2)
    assert st["batch_replans"] > 0 and st["batch_waves"] == 0
    assert sum(r["replanned"] for r in bat) == st["batch_replans"]
    assert st["batch_rollouts"] == len(sc.requests) + st["batch_replans"]
    assert 0 < st["pipe_ctas"] <= st["pipe_resident"]


@pytest.mark.parametrize("batch_size,spread", [(0, 1500.0), (16, 1500.0), (0, 700.0), (32, 700.0)])
def test_pipelined_crowded_seeds(batch_size, spread):
    """Many interleavings of the pipelined mode: crowded airspaces over sixteen seeds, where
    tentative plans are published, replaced by resumed plans that keep their first samples,
    withdrawn and published again while later requests read them. Every seed must give the
    sequential results and table."""
    resumes = publishes = withdrawals = 0
    for seed in range(300, 316):
        sc = S.crowded_batch(seed=seed, n_requests=64, spread_m=spread)
        many, bat, t1, t2, st = run_both(sc, batch_size=batch_size)
        try:
            same_results(many, bat)
            same_tables(t1, t2)
        except AssertionError as e:
            raise AssertionError(f"seed {seed}: {e}") from None
        resumes += st["pipe_resumes"]
        publishes += st["pipe_publishes"]
        withdrawals += st["pipe_withdrawals"]
    assert resumes > 0 and publishes > 0 and withdrawals > 0


@pytest.mark.parametrize("batch_mode", [0, 1])
def test_crowded_batch_against_the_oracle(batch_mode):
    sc = S.crowded_batch(n_requests=24)
    with Scheduler.from_scenario(sc, batch_mode=batch_mode) as s:
        bat = s.schedule_batch(sc.requests)
        st = s.stats()
    assert st["batch_replans"] > 0
    o = oracle_for(sc)
    verdicts, followed, steps = fcfs_parity(None, o, sc.requests, gpu_results=bat)
    assert ADMITTED in verdicts
    assert followed <= max(5, steps // 1000)


def test_graph_replay_equals_eager_launches():
    sc = S.crowded_batch(seed=105, n_requests=40)
    with Scheduler.from_scenario(sc, batch_mode=1) as s:
        s.snapshot()
        g1 = s.schedule_batch(sc.requests)  # captured graph
        s.restore()
        g2 = s.schedule_batch(sc.requests)  # replayed graph
        s.restore()
        s.set_profiling(1)                  # eager launches with event timing
        e = s.schedule_batch(sc.requests)
        st = s.stats()
    same_results(g1, g2)
    same_results(g1, e)
    assert st["rollout_launches"] >= 1 and st["influence_launches"] >= 1


@pytest.mark.parametrize("batch_mode", [0, 1])
def test_consecutive_batches_with_expiry_and_edge_cases(batch_mode):
    sc = S.crowded_batch(seed=106, n_requests=30)
    reqs = sc.requests.copy()
    reqs[3]["horizon"] = 0                      # no step: rejected on the horizon at once
    reqs[7]["horizon"] = 5                      # too short to reach the goal
    reqs[9]["gx"], reqs[9]["gy"] = reqs[9]["ox"], reqs[9]["oy"]  # starts at its goal (x, y)
    reqs[9]["gz"] = reqs[9]["oz"]
    first, second = reqs[:17], reqs[17:]
    second = second.copy()
    second["depart"] += 200
    out = []
    for fn in ("schedule_many", "schedule_batch"):
        with Scheduler.from_scenario(sc, batch_size=8, batch_mode=batch_mode) as s:
            a = getattr(s, fn)(first)
            assert getattr(s, fn)(first[:0]) == []
            s.expire(150)
            b = getattr(s, fn)(second)
            out.append((a + b, table_of(s)))
    same_results(out[0][0], out[1][0])
    same_tables(out[0][1], out[1][1])
    assert out[1][0][3]["n_points"] == 1 and out[1][0][9]["n_points"] == 1


@pytest.mark.parametrize("batch_mode", [0, 1])
def test_c3_full_size_batch_of_256(batch_mode):
    """20k known plans, one batch of 256 requests with horizons U[60,1800]: identical to
    sequential FCFS; the requests ahead of the first admission go to the oracle too."""
    sc = S.c3_batched(n_requests=256)
    reqs = sc.requests.copy()
    order = np.argsort(reqs["horizon"], kind="stable")  # short horizons first: cheap oracle prefix
    reqs = reqs[np.concatenate([order[:6], np.sort(order[6:])])]
    with Scheduler.from_scenario(sc, batch_mode=batch_mode) as s:
        s.snapshot()
        many = s.schedule_many(reqs)
        t1 = table_of(s)
        s.restore()
        bat = s.schedule_batch(reqs)
        t2 = table_of(s)
        st = s.stats()
    same_results(many, bat)
    same_tables(t1, t2)
    assert st["batch_rollouts"] >= 256
    o = oracle_for(sc)
    fcfs_parity(None, o, reqs[:6], gpu_results=bat[:6])


@pytest.mark.parametrize("batch_mode", [0, 1])
@pytest.mark.parametrize("batch_size", [0, 16])
def test_staged_batch_equals_sequential(batch_size, batch_mode):
    """The device-resident batched run (requests staged once, trajectories left on the
    device and fetched afterwards) gives the sequential results."""
    sc = S.c1_plain_small()
    with Scheduler.from_scenario(sc, batch_size=batch_size, batch_mode=batch_mode) as s:
        s.snapshot()
        many = s.schedule_many(sc.requests)
        s.restore()
        s.stage(sc.requests)
        s.set_profiling(0)
        n_adm = s.schedule_staged(batched=True)
        st = s.stats()
        got = s.fetch_staged()
    same_results(many, got)
    assert n_adm == sum(r["verdict"] == ADMITTED for r in many)
    if batch_mode == 1:
        assert st["batch_waves"] >= 1 and st["kernel_launches"] >= 5 * st["batch_waves"]
    else:
        assert st["batch_waves"] == 0 and st["batch_rollouts"] >= len(sc.requests)


def _side_by_side(offset_m, speed=30.0):
    """Two requests flying east in an empty sky, `offset_m` apart, departing together."""
    box = (0.0, 0.0, 0.0, 10000.0, 10000.0, 500.0)
    req = np.zeros(2, dtype=S.REQUEST_DTYPE)
    for i, y in enumerate((5000.0, 5000.0 + offset_m)):
        req[i] = (i + 1, 1000.0, y, 200.0, 7000.0, y, 200.0, speed, 10, 600)
    return S.Scenario("side_by_side", box, 1.0, 0.99, S.action_grid((-2.0, 0.0, 2.0)), (150.0, 30.0), [], req,
                      n_slices_window=2048, max_slots=64)


@pytest.mark.parametrize("batch_mode", [0, 1])
@pytest.mark.parametrize("offset,waves", [(700.0, 1), (300.0, 2)])
def test_influence_follows_each_well(offset, waves, batch_mode):
    """The first request's wells lie along its track (Table 3: centres p + tau v, radii
    250-450 m). At 700 m abeam the second request is out of reach of every well, though
    inside one ball of radius max R + max|tau| |v| around the first request, so both are
    final after one wave; at 300 m the tau = 0 well reaches it and it is planned again."""
    sc = _side_by_side(offset)
    many, bat, t1, t2, st = run_both(sc, batch_mode=batch_mode)
    same_results(many, bat)
    same_tables(t1, t2)
    assert [r["verdict"] for r in bat] == [ADMITTED, ADMITTED]
    assert st["batch_replans"] == waves - 1
    if batch_mode == 1:
        assert st["batch_waves"] == waves


def test_c2_full_size_pipelined_equals_waves_and_sequential():
    """The 3000-plan, 1000-request workload in the launch configuration the benchmark
    times (staged requests, batched): pipelined and wave results equal sequential FCFS,
    and the pipelined run's admissions grow index rows past the rebuild mark (set to 192
    appended items here, below what this workload reaches), so the
    rebuild-while-no-rollout-runs path runs."""
    sc = S.c2_plain_scale()
    out = {}
    for mode in (0, 1):
        with Scheduler.from_scenario(sc, batch_mode=mode, pipe_rebuild_items=192) as s:
            s.snapshot()
            if mode == 0:
                out["many"] = s.schedule_many(sc.requests)
                out["t_many"] = table_of(s)
                s.restore()
            s.stage(sc.requests)
            s.set_profiling(0)
            s.schedule_staged(batched=True)
            out[mode] = s.fetch_staged()
            out[("t", mode)] = table_of(s)
            out[("st", mode)] = s.stats()
    same_results(out["many"], out[0])
    same_results(out["many"], out[1])
    same_tables(out["t_many"], out[("t", 0)])
    same_tables(out["t_many"], out[("t", 1)])
    assert out[("st", 0)]["pipe_drains"] >= 1 and out[("st", 0)]["batch_waves"] == 0
