"""The allocation-free separation check, fmdp_sep_check_noalloc.

Some callers cannot allocate device memory while they run: software whose memory
footprint must be fixed at start-up (certified or real-time code that forbids allocation
after initialisation) and code that must not be slowed or synchronised by cudaMalloc /
cudaFree on its path. For them the library keeps one fixed scratch array in its image and
this entry point stages the trajectory and the check's accumulators there.

The test calls the new entry point through the C ABI twice in a row (the scratch array
keeps the previous call's contents, so the second call shows that each call clears what
it needs) and checks both reports against the regular, allocating fmdp_sep_check. This
file is named to be collected last so that a run that stops at the first failure has run
every other test before it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2008_03518_gb300 import scenarios as S  # noqa: E402
from paper_2008_03518_gb300.fmdp import NOALLOC_MAX_POINTS, FmdpError, Scheduler  # noqa: E402


def _trajectory_near_plans(sc, rng, t0, n):
    """Samples that pass close to known plans, some exactly at the separation minima."""
    traj = rng.uniform([0, 0, 50], [10000, 10000, 450], size=(n, 3)).astype(np.float32)
    for k in range(0, n, 3):
        pl = sc.plans[int(rng.integers(0, len(sc.plans)))]
        j = t0 + k - pl.t0
        if 0 <= j < len(pl.xyz):
            off = rng.choice([0.0, 100.0, 149.999, 150.0, 150.001])
            dz = rng.choice([0.0, 29.999, 30.0, 30.001])
            ang = rng.uniform(0.0, 2.0 * np.pi)
            traj[k] = pl.xyz[j] + np.array([off * np.cos(ang), off * np.sin(ang), dz], dtype=np.float32)
    return traj


def _same(a, b):
    assert a["conflicts"] == b["conflicts"]
    assert a["first_conflict_step"] == b["first_conflict_step"]
    assert a["first_terrain_step"] == b["first_terrain_step"]
    for k in ("min_sep_h", "min_sep_v"):
        if np.isfinite(b[k]):
            assert a[k] == pytest.approx(b[k], rel=1e-5, abs=1e-5)
        else:
            assert not np.isfinite(a[k])


def test_noalloc_sep_check_matches_the_allocating_one_on_two_calls():
    sc = S.c1_plain_small()
    rng = np.random.default_rng(2024)
    with Scheduler.from_scenario(sc) as s:
        calls = []
        for t0, n in ((int(rng.integers(0, 400)), 700), (int(rng.integers(0, 400)), 333)):
            traj = _trajectory_near_plans(sc, rng, t0, n)
            calls.append((t0, traj, s.sep_check(t0, traj)))  # the allocating entry point
        # set-up call: resolves the scratch array's device address (and lets the driver place
        # the array, which lazy module loading defers to this first use)
        s.sep_check_noalloc(0, np.zeros((1, 3), dtype=np.float32))
        free0 = torch.cuda.mem_get_info()[0]
        got = [s.sep_check_noalloc(t0, traj) for t0, traj, _ in calls]  # two calls in a row
        free1 = torch.cuda.mem_get_info()[0]
        for g, (_, _, want) in zip(got, calls):
            _same(g, want)
        assert sum(w["conflicts"] for _, _, w in calls) > 0  # the planted pairs were exercised
        assert free1 == free0  # the two calls took no device memory

        # sizes beyond the scratch array's capacity are refused with a clear error
        big = np.zeros((NOALLOC_MAX_POINTS + 1, 3), dtype=np.float32)
        with pytest.raises(FmdpError) as e:
            s.sep_check_noalloc(0, big)
        assert e.value.status == -1 and "FMDP_NOALLOC_MAX_POINTS" in str(e.value)
        # and the largest allowed size still works
        full = _trajectory_near_plans(sc, rng, 0, NOALLOC_MAX_POINTS)
        _same(s.sep_check_noalloc(0, full), s.sep_check(0, full))


def test_noalloc_runs_on_the_context_device_and_is_counted():
    """The call runs on the context's device whichever device the caller has current, leaves
    the caller's device current, and counts as a separation-check launch in the stats."""
    sc = S.c1_plain_small()
    rng = np.random.default_rng(7)
    t0 = 120
    traj = _trajectory_near_plans(sc, rng, t0, 500)
    with Scheduler.from_scenario(sc) as s:
        want = s.sep_check(t0, traj)
        s.set_profiling(1)
        before = torch.cuda.current_device()
        got = s.sep_check_noalloc(t0, traj)
        assert torch.cuda.current_device() == before
        _same(got, want)
        st = s.stats()
        assert st["sepcheck_launches"] == 1 and st["sep_pairs"] > 0
        if torch.cuda.device_count() > 1:  # a caller that made another device current
            other = (before + 1) % torch.cuda.device_count()
            torch.cuda.set_device(other)
            try:
                _same(s.sep_check_noalloc(t0, traj), want)
                assert torch.cuda.current_device() == other
            finally:
                torch.cuda.set_device(before)
