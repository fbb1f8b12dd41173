"""The lookahead window W (Sec. IV "Forward project", Alg. 9) on the GPU against the FP64
oracle (whose window is pinned in test_oracle_lookahead.py): per-action values within
1e-5 of the term scale, the same actions except at near-ties (where the oracle follows
the GPU), bit-identical trajectories and verdicts under FCFS.

- the paper's own fidelity: W = 10 sub-steps of dt = 0.1 s (the e1_fine scenario);
- W = 2 and 4 at dt = 1 s on C1 traffic, MAX and SUM;
- terrain clearance and static wells along the window;
- batched calls with W > 1 (speculative waves of lookahead rollouts, re-plans included)
  give the sequential results; entry points that need W = 1
  refuse W > 1.
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
from tests.parity_util import fcfs_parity  # noqa: E402

from test_gpu_batch import same_results, same_tables, table_of  # noqa: E402


def _pair(sc, W, **kw):
    return Scheduler.from_scenario(sc, lookahead_W=W, **kw), Oracle.from_scenario(sc, lookahead_W=W, **kw)


def test_paper_fidelity_w10_dt01_lockstep_and_fcfs():
    sc = S.e1_fine()
    s, o = _pair(sc, sc.meta["lookahead_W"])
    with s:
        verdicts, followed, steps = fcfs_parity(s, o, sc.requests[:6], trace_q=True)
    assert steps > 3000 and ADMITTED in verdicts
    # at 0.1 s the actions of a step differ by metres, so mirror-image actions (left and
    # right turns around a well ahead, climbs around the goal altitude) tie exactly in
    # exact arithmetic and rounding picks one: both sides flag these steps as near-ties
    assert followed <= steps // 20


@pytest.mark.parametrize("W,combine", [(2, 0), (4, 0), (4, 1)])
def test_c1_windows_lockstep_and_fcfs(W, combine):
    sc = S.c1_plain_small()
    s, o = _pair(sc, W, combine=combine)
    with s:
        verdicts, followed, steps = fcfs_parity(s, o, sc.requests[:8], trace_q=True)
    assert steps > 1000 and ADMITTED in verdicts


def test_terrain_and_static_wells_along_the_window():
    sc = S.c2_plain_scale(n_plans=300, n_requests=6)
    sw = np.array([[15000.0, 15000.0, 300.0, 2000.0, 1000.0, 0.99],
                   [8000.0, 22000.0, 200.0, 1500.0, 1000.0, 0.99]])
    sc.static_wells = sw
    s, o = _pair(sc, 3)
    with s:
        verdicts, followed, steps = fcfs_parity(s, o, sc.requests[:4], trace_q=True)
    assert steps > 500


@pytest.mark.parametrize("W", [3, 10])
def test_batched_window_rollouts_replan_and_equal_sequential(W):
    """Speculative waves of lookahead rollouts: crossing paths force re-plans, and the
    results and the table equal planning one request at a time."""
    sc = S.crowded_batch(seed=141, n_requests=32)
    with Scheduler.from_scenario(sc, lookahead_W=W) as s:
        a = s.schedule_many(sc.requests)
        ta = table_of(s)
    with Scheduler.from_scenario(sc, lookahead_W=W) as s:
        b = s.schedule_batch(sc.requests)
        st = s.stats()
        tb = table_of(s)
    same_results(a, b)
    same_tables(ta, tb)
    assert st["batch_replans"] > 0 and st["batch_waves"] > 1


def test_batched_paper_fidelity_w10_dt01_equals_sequential():
    sc = S.e1_fine()
    with Scheduler.from_scenario(sc, lookahead_W=10) as s:
        a = s.schedule_many(sc.requests)
    with Scheduler.from_scenario(sc, lookahead_W=10) as s:
        s.stage(sc.requests)
        s.schedule_staged(batched=True)
        b = s.fetch_staged()
    same_results(a, b)


def test_batched_calls_with_a_window_equal_sequential():
    sc = S.c1_plain_small()
    with Scheduler.from_scenario(sc, lookahead_W=3) as s:
        a = s.schedule_many(sc.requests[:10])
    with Scheduler.from_scenario(sc, lookahead_W=3) as s:
        b = s.schedule_batch(sc.requests[:10])
    same_results(a, b)
    with Scheduler.from_scenario(sc, lookahead_W=3) as s:
        with pytest.raises(FmdpError):
            s.serve(sc.requests[:4], np.zeros(4))
        with pytest.raises(FmdpError):
            s.schedule_departures(sc.requests[:2], [0, 10])
        with pytest.raises(FmdpError):
            s.autotune(sc.requests[:4])
    with pytest.raises(FmdpError):
        Scheduler.from_scenario(sc, lookahead_W=17)
