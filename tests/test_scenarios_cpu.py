"""The seeded input generators against the recipe they promise (CPU).

The parity tests and the benchmark run on synthetic airspaces shaped like the paper's
workloads. These checks tie each generator to its stated shape: counts, boxes, time steps,
speed, altitude and departure ranges, sample spacing (one point per speed x dt of arc),
terrain clearance of request endpoints, the action sets, and determinism under a seed.
"""
import numpy as np

from paper_2008_03518_gb300 import scenarios as S


def spacing_ok(xyz, v_lo, v_hi, dt):
    """Consecutive samples are one speed x dt apart (the last one may be shorter)."""
    if len(xyz) < 3:
        return True
    d = np.linalg.norm(np.diff(np.asarray(xyz, dtype=np.float64), axis=0), axis=1)[:-1]
    v = d / dt
    return bool(np.all(v >= v_lo - 1e-2) and np.all(v <= v_hi + 1e-2) and np.ptp(v) < 1e-2 * max(v.max(), 1.0))


def in_box(xyz, box, tol=1e-3):
    xyz = np.asarray(xyz)
    return bool(np.all(xyz[:, 0] >= box[0] - tol) and np.all(xyz[:, 0] <= box[3] + tol)
                and np.all(xyz[:, 1] >= box[1] - tol) and np.all(xyz[:, 1] <= box[4] + tol)
                and np.all(xyz[:, 2] >= box[2] - tol) and np.all(xyz[:, 2] <= box[5] + tol))


def test_c1_plain_small():
    sc = S.c1_plain_small()
    assert sc.box == (0.0, 0.0, 0.0, 10000.0, 10000.0, 500.0) and sc.dt == 1.0 and sc.gamma == 0.99
    assert sc.sep == (150.0, 30.0) and len(sc.plans) == 200 and len(sc.requests) == 50
    assert sorted({a[0] for a in sc.actions}) == [-30.0, -15.0, 0.0, 15.0, 30.0]
    assert sorted({a[1] for a in sc.actions}) == [-2.0, 0.0, 2.0] and len(sc.actions) == 15
    for p in sc.plans:
        assert 0 <= p.t0 <= 600 and in_box(p.xyz, sc.box)
        assert np.all((p.xyz[:, 2] >= 50.0 - 1e-3) & (p.xyz[:, 2] <= 450.0 + 1e-3))
        assert spacing_ok(p.xyz, 20.0, 40.0, 1.0)
    r = sc.requests
    assert np.all(r["horizon"] == 1200) and np.all((r["depart"] >= 0) & (r["depart"] <= 600))
    assert np.all((r["speed"] >= 20.0) & (r["speed"] <= 40.0))
    for k in ("oz", "gz"):
        assert np.all((r[k] >= 50.0) & (r[k] <= 450.0))


def test_c2_plain_scale_terrain_and_legs():
    sc = S.c2_plain_scale()
    hm = sc.heightmap
    assert hm.shape == (512, 512) and hm.dtype == np.float32
    assert hm.min() >= 0.0 and hm.max() <= 300.0 and hm.max() > 200.0  # the stated [0, 300] m
    assert sc.clearance == 60.0 and len(sc.plans) == 3000 and len(sc.requests) == 1000
    assert sorted({a[1] for a in sc.actions}) == [-4.0, -2.0, 0.0, 2.0, 4.0] and len(sc.actions) == 25
    r = sc.requests
    assert np.all(r["horizon"] == 1800) and np.all((r["depart"] >= 0) & (r["depart"] <= 1800))
    for i in range(0, 1000, 37):  # endpoints at the cell's highest node + U[60, 500] m (or below the top)
        for x, y, z in ((r["ox"][i], r["oy"][i], r["oz"][i]), (r["gx"][i], r["gy"][i], r["gz"][i])):
            base = S._cell_max(hm, sc.box, x, y)
            assert (60.0 - 1e-6 <= z - base <= 500.0 + 1e-6) or z == sc.box[5] - 1.0
    for p in sc.plans[::50]:
        assert 0 <= p.t0 <= 1800 and in_box(p.xyz, sc.box)
        # a multi-leg polyline: one sample per speed x dt of arc, so chords are at most that
        d = np.linalg.norm(np.diff(p.xyz.astype(np.float64), axis=0), axis=1)
        assert d.max() <= 40.0 + 1e-2 and len(p.xyz) > 3000.0 / 40.0 * 3


def test_c3_horizons_and_reach():
    sc = S.c3_batched(n_plans=2000)  # the plan count does not change the requests' recipe
    r = sc.requests
    assert len(r) == 1024 and r["horizon"].min() >= 60 and r["horizon"].max() <= 1800
    L = np.hypot(r["gx"] - r["ox"], r["gy"] - r["oy"])
    want = 0.8 * r["speed"] * r["horizon"]
    assert np.all(L <= want + 1e-6)  # clipping into the box only shortens the leg
    assert np.mean(np.abs(L - want) < 1e-6 * np.maximum(want, 1.0)) > 0.3  # most are not clipped


def test_e1_fine_paper_fidelity():
    sc = S.e1_fine()
    assert sc.dt == 0.1 and sc.meta["lookahead_W"] == 10 and len(sc.plans) == 60 and len(sc.requests) == 12
    for p in sc.plans:
        assert 0 <= p.t0 <= 600 and spacing_ok(p.xyz, 20.0, 40.0, 0.1)  # departures within 60 s
        assert np.all((p.xyz[:, 2] >= 100.0 - 1e-3) & (p.xyz[:, 2] <= 400.0 + 1e-3))
    assert np.all(sc.requests["horizon"] == 3000)  # 300 s


def test_crowded_batch_crossing_geometry():
    sc = S.crowded_batch()
    r = sc.requests
    o = np.hypot(r["ox"] - 5000.0, r["oy"] - 5000.0)
    g = np.hypot(r["gx"] - 5000.0, r["gy"] - 5000.0)
    assert np.all(o <= 1500.0 + 1e-6) and np.all((g >= 3000.0 - 1e-6) & (g <= 4500.0 + 1e-6))
    assert np.all((r["depart"] >= 0) & (r["depart"] <= 30))


def test_generators_are_deterministic_under_their_seeds():
    a, b = S.c1_plain_small(), S.c1_plain_small()
    assert np.array_equal(a.requests, b.requests)
    assert all(p.t0 == q.t0 and np.array_equal(p.xyz, q.xyz) for p, q in zip(a.plans, b.plans))
    assert not np.array_equal(S.c1_plain_small(seed=7).requests, a.requests)
    h1, h2 = S.fractal_heightmap(5, n=64), S.fractal_heightmap(5, n=64)
    assert np.array_equal(h1, h2)
