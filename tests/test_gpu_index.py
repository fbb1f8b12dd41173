"""The spatial index of the plan table against the full scan.

A rollout step with the index reads only the plan samples whose cell lies within the
query radius of the state (plus the extra list); the full scan reads every slot. Both
apply the same cull and the same arithmetic to the plans within reach, and every other
plan adds an exact zero to the action values, so trajectories, action values and verdicts
must agree bit for bit. The tests also keep the index in step with the table through
every operation that changes it (bulk and single additions, admissions, expiry, snapshot
and restore, clear), and force the paths for fast plans (the extra list) and for
neighbourhoods larger than the shared-memory staging buffer (reads from global memory).
The oracle parity tests in test_gpu_parity.py run with the index (the default).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import ADMITTED, Oracle  # noqa: E402
from paper_2008_03518_gb300 import scenarios as S  # noqa: E402
from paper_2008_03518_gb300.fmdp import Scheduler  # noqa: E402

from parity_util import fcfs_parity  # noqa: E402
from test_gpu_batch import same_results, same_tables, table_of  # noqa: E402


def both(sc, **kw):
    return Scheduler.from_scenario(sc, full_scan=True, **kw), Scheduler.from_scenario(sc, **kw)


def test_traces_equal_full_scan_c1():
    sc = S.c1_plain_small()
    full, idx = both(sc)
    with full, idx:
        for r in sc.requests[:8]:
            a, b = full.rollout_trace(r), idx.rollout_trace(r)
            np.testing.assert_array_equal(a["xyz"], b["xyz"])
            np.testing.assert_array_equal(a["q"], b["q"])
            np.testing.assert_array_equal(a["actions"], b["actions"])


@pytest.mark.parametrize("combine", [0, 1])
def test_fcfs_equal_full_scan_c1(combine):
    sc = S.c1_plain_small()
    full, idx = both(sc, combine=combine)
    with full, idx:
        a = full.schedule_many(sc.requests)
        b = idx.schedule_many(sc.requests)
        same_results(a, b)
        same_tables(table_of(full), table_of(idx))
    assert sum(r["verdict"] == ADMITTED for r in b) > 0


def test_terrain_static_wells_equal_full_scan():
    from test_gpu_parity import _terrain_scenario

    sc = _terrain_scenario()
    full, idx = both(sc)
    with full, idx:
        same_results(full.schedule_many(sc.requests), idx.schedule_many(sc.requests))


def test_c2_subset_sequential_and_batched_equal_full_scan():
    sc = S.c2_plain_scale(n_requests=48)
    full, idx = both(sc)
    with full, idx:
        idx.set_profiling(1)
        a = full.schedule_many(sc.requests)
        b = idx.schedule_batch(sc.requests)
        st = idx.stats()
        same_results(a, b)
        same_tables(table_of(full), table_of(idx))
    # the index reads far fewer plan samples than the slots a full scan streams
    assert 0 < st["items_scanned"] < 0.2 * st["slots_scanned"]


def test_index_follows_every_table_change():
    sc = S.crowded_batch(seed=107, n_requests=36)
    full, idx = both(sc, batch_size=12)
    with full, idx:
        out = []
        for s in (full, idx):
            got = []
            s.snapshot()
            got += s.schedule_many(sc.requests[:10])
            # single additions (appended to the rows' extra lists), one of them fast
            for k in range(3):
                got.append(s.add_plan(*_straight(sc, k, fast=(k == 1))))
            got += s.schedule_batch(sc.requests[10:22])
            s.expire(60)
            got += s.schedule_many(_shift(sc.requests[22:30], 100))
            s.restore()
            got += s.schedule_batch(sc.requests[:12])
            s.clear()
            s.add_plans([(p.t0, p.xyz) for p in sc.plans[:80]])
            got += s.schedule_many(sc.requests[12:20])
            out.append((got, table_of(s)))
        ga, gb = out[0][0], out[1][0]
        assert len(ga) == len(gb)
        for x, y in zip(ga, gb):
            if isinstance(x, dict):
                same_results([x], [y])
            else:
                assert x == y
        same_tables(out[0][1], out[1][1])


def _straight(sc, k, fast=False):
    """A straight plan through the middle of the crowded region (fast: 120 m/s)."""
    v = 120.0 if fast else 30.0
    n = 300
    t = np.arange(n, dtype=np.float64)
    ang = 0.7 + 1.3 * k
    x = 5000.0 - 0.5 * v * n * np.cos(ang) + v * t * np.cos(ang)
    y = 5000.0 - 0.5 * v * n * np.sin(ang) + v * t * np.sin(ang)
    z = np.full(n, 200.0 + 40.0 * k)
    xyz = np.stack([x, y, z], axis=1).astype(np.float32)
    return 5 + 7 * k, np.clip(xyz, 0.0, 10000.0).astype(np.float32)


def _shift(reqs, dt):
    r = reqs.copy()
    r["depart"] += dt
    return r


@pytest.mark.parametrize("stage_items", [32, 200])
def test_staging_overflow_reads_global_memory(stage_items):
    """Neighbourhoods larger than the staging buffer: the rest is read from the index."""
    sc = S.crowded_batch(seed=108, n_plans=600, n_requests=20)
    full = Scheduler.from_scenario(sc, full_scan=True)
    idx = Scheduler.from_scenario(sc, index_stage_items=stage_items)
    with full, idx:
        same_results(full.schedule_many(sc.requests), idx.schedule_many(sc.requests))


def test_fast_plans_in_the_extra_list_against_the_oracle():
    """Known plans faster than the index's speed bound are read at every step; with a low
    bound most plans take that path, and the result still matches the oracle."""
    sc = S.c1_plain_small()
    sc.requests = sc.requests[:10]
    with Scheduler.from_scenario(sc, index_vmax_mps=25.0) as s:
        o = Oracle.from_scenario(sc)
        fcfs_parity(s, o, sc.requests, trace_q=True)


def test_a_later_scheduler_with_a_smaller_index_leaves_the_earlier_one_working():
    """Kernel attributes are shared by every scheduler of a process: creating one with a
    smaller index grid must not shrink the shared memory the earlier one launches with."""
    big = S.c2_plain_scale(n_plans=300, n_requests=4)
    with Scheduler.from_scenario(big) as s1:
        s1.snapshot()
        small = S.c1_plain_small()
        with Scheduler.from_scenario(small) as s2:
            s2.schedule(small.requests[0])
        s1.restore()  # rebuilds every index row of the larger grid
        res = s1.schedule_many(big.requests[:2])
    assert len(res) == 2
