"""The plan table to a file and back (fmdp_save_plans / fmdp_load_plans): the accepted-plan
database that Sec. V keeps across scheduling runs, loaded at start and appended to.

A table saved after some admissions and loaded into an emptied context holds the same plans
(first step and every sample, bit for bit), and the requests planned after it get the same
results as on the original table. A file that is not a whole plan file is refused with
FMDP_ERR_IO and leaves the table as it was.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2008_03518_gb300 import scenarios as S  # noqa: E402
from paper_2008_03518_gb300.fmdp import FmdpError, Scheduler  # noqa: E402

KEYS = ("verdict", "n_points", "first_conflict_step", "first_terrain_step", "near_ties", "min_sep_h", "min_sep_v")


def plans_of(s):
    """The table's plans as (first step, samples), in an order that does not depend on ids."""
    out = [s.get_plan(i) for i in s.query_plans(-(1 << 40), 1 << 40)]
    return sorted(out, key=lambda p: (p[0], p[1].tobytes()))


def same_plans(a, b):
    assert len(a) == len(b)
    for (ta, xa), (tb, xb) in zip(a, b):
        assert ta == tb
        np.testing.assert_array_equal(xa, xb)


def same_results(a, b):
    assert len(a) == len(b)
    for i, (x, y) in enumerate(zip(a, b)):
        for k in KEYS:
            assert x[k] == y[k] or (np.isnan(x[k]) and np.isnan(y[k])), (i, k, x[k], y[k])
        np.testing.assert_array_equal(x["xyz"], y["xyz"], err_msg=f"request {i}")
        np.testing.assert_array_equal(x["actions"], y["actions"], err_msg=f"request {i}")


def test_saved_table_loads_back_and_plans_the_same(tmp_path):
    sc = S.c1_plain_small()
    path = str(tmp_path / "plans.fmdp")
    with Scheduler.from_scenario(sc) as s:
        first = s.schedule_many(sc.requests[:20])
        assert any(r["verdict"] == 0 for r in first)
        saved = plans_of(s)
        assert s.save_plans(path) == len(saved)
        later = s.schedule_many(sc.requests[20:40])
    with Scheduler.from_scenario(sc) as s2:
        s2.clear()
        assert plans_of(s2) == []
        ids = s2.load_plans(path)
        assert len(ids) == len(saved) and len(set(ids.tolist())) == len(ids)
        same_plans(plans_of(s2), saved)
        same_results(later, s2.schedule_many(sc.requests[20:40]))


def test_loading_into_an_empty_table_takes_the_saved_window(tmp_path):
    """A table whose window has moved (expiry to step 300) loads into a fresh context, whose
    window starts earlier, with every plan where it was; a plan that started before the
    window is saved, and loaded, from the window's first step."""
    sc = S.c1_plain_small()
    path = str(tmp_path / "moved.fmdp")
    with Scheduler.from_scenario(sc) as s:
        s.expire(300)
        ids = s.query_plans(-(1 << 40), 1 << 40)
        whole, clipped = [], 0
        for i in ids:
            try:
                whole.append(s.get_plan(i))
            except FmdpError as e:  # started before the window: not readable whole
                assert e.status == -6
                clipped += 1
        assert whole and clipped > 0
        assert s.save_plans(path) == len(ids)
    with Scheduler.from_scenario(sc) as s2:
        s2.clear()
        s2.load_plans(path)
        loaded = plans_of(s2)
        assert len(loaded) == len(ids)
        assert sum(1 for t, _ in loaded if t == 300) >= clipped
        keys = {(t, x.tobytes()) for t, x in loaded}
        assert all((t, x.tobytes()) in keys for t, x in whole)


def test_a_broken_file_is_refused_and_changes_nothing(tmp_path):
    sc = S.c1_plain_small()
    good = tmp_path / "good.fmdp"
    with Scheduler.from_scenario(sc) as s:
        s.save_plans(str(good))
        before = plans_of(s)
        data = good.read_bytes()
        for name, blob in (("garbage", b"not a plan file at all" * 4), ("truncated", data[: len(data) // 2]),
                           ("empty", b"")):
            p = tmp_path / name
            p.write_bytes(blob)
            with pytest.raises(FmdpError) as e:
                s.load_plans(str(p))
            assert e.value.status == -8
        with pytest.raises(FmdpError) as e:
            s.load_plans(str(tmp_path / "missing.fmdp"))
        assert e.value.status == -8
        same_plans(plans_of(s), before)
