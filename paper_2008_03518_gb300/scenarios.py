"""Seeded synthetic airspaces for FastMDP first-come-first-served planning.

This module makes INPUTS only: airspace boxes, fractal heightmaps, known flight
plans sampled along straight or multi-leg routes, and planning requests. It holds
none of the planner's arithmetic (no values, wells, forward projection, argmax or
separation test), so the FP64 oracle and the CUDA scheduler can both consume its
output without sharing any of the method.

The paper's own scenario, terrain and accepted-plan database are not published
(Sec. V keeps the database "in a file"; Sec. VII hopes to release it), so these
generators stand in for them with the shapes of the paper's workloads:
  * known plans are lists of trajectory points, one per time step (Sec. V: plans
    are stored "in the form of trajectory points");
  * the actions are a heading-change x climb-rate grid (Sec. IV, forward projection
    over an action set, as in the paper's Alg. 1 "aircraft actions (precomputed)");
  * terrain is a heightmap plus optional manually-placed restricted-volume wells
    (Table 3, terrain row).

Randomness is numpy's PCG64 (``numpy.random.default_rng(seed)``), which is
platform independent; every float that leaves this module is produced by basic
IEEE operations, so x86 and aarch64 hosts produce identical scenarios.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

# Heading-change set (degrees) used by every workload: five headings 15 deg apart.
HEADINGS_DEG = (-30.0, -15.0, 0.0, 15.0, 30.0)


@dataclass
class Plan:
    """A known flight plan: one fp32 (x, y, z) point per time step from t0."""
    t0: int
    xyz: np.ndarray  # float32 [n, 3]


@dataclass
class Scenario:
    name: str
    box: Tuple[float, float, float, float, float, float]  # x0, y0, z0, x1, y1, z1
    dt: float
    gamma: float
    actions: List[Tuple[float, float]]  # (heading change deg, climb m/s), index order
    sep: Tuple[float, float]  # horizontal, vertical minima (m)
    plans: List[Plan]
    requests: np.ndarray  # structured, REQUEST_DTYPE
    heightmap: Optional[np.ndarray] = None  # float32 [ny, nx] or None
    clearance: float = 0.0
    goal_reward: float = 200.0
    static_wells: Optional[np.ndarray] = None  # float64 [n, 6]: x, y, z, R, |r|, gamma
    n_slices_window: int = 4096
    max_slots: int = 0
    meta: dict = field(default_factory=dict)


REQUEST_DTYPE = np.dtype([
    ("req_id", np.uint64),
    ("ox", np.float64), ("oy", np.float64), ("oz", np.float64),
    ("gx", np.float64), ("gy", np.float64), ("gz", np.float64),
    ("speed", np.float64),
    ("depart", np.int64),
    ("horizon", np.int32),
])


def action_grid(climbs):
    """Heading-major action list: 5 heading changes x len(climbs) climb rates."""
    return [(h, c) for h in HEADINGS_DEG for c in climbs]


# ---------------------------------------------------------------------------
# terrain


def diamond_square(rng: np.random.Generator, n_pow: int = 9, roughness: float = 0.55) -> np.ndarray:
    """Fractal heightmap on a (2^n + 1)^2 grid by the diamond-square method.

    Returns float64 values; the caller crops and rescales.
    """
    size = (1 << n_pow) + 1
    h = np.zeros((size, size), dtype=np.float64)
    corners = rng.uniform(-1.0, 1.0, size=4)
    h[0, 0], h[0, -1], h[-1, 0], h[-1, -1] = corners
    step = size - 1
    amp = 1.0
    while step > 1:
        half = step // 2
        # diamond step: centres of squares
        ys = np.arange(half, size, step)
        xs = np.arange(half, size, step)
        yy, xx = np.meshgrid(ys, xs, indexing="ij")
        avg = (h[yy - half, xx - half] + h[yy - half, xx + half]
               + h[yy + half, xx - half] + h[yy + half, xx + half]) * 0.25
        h[yy, xx] = avg + rng.uniform(-amp, amp, size=avg.shape)
        # square step: edge midpoints (rows alternate their x offset)
        for y in range(0, size, half):
            x_start = half if (y // half) % 2 == 0 else 0
            xs2 = np.arange(x_start, size, step)
            acc = np.zeros(xs2.size)
            cnt = np.zeros(xs2.size)
            if y - half >= 0:
                acc += h[y - half, xs2]; cnt += 1
            if y + half < size:
                acc += h[y + half, xs2]; cnt += 1
            m = xs2 - half >= 0
            acc[m] += h[y, xs2[m] - half]; cnt[m] += 1
            m = xs2 + half < size
            acc[m] += h[y, xs2[m] + half]; cnt[m] += 1
            h[y, xs2] = acc / cnt + rng.uniform(-amp, amp, size=xs2.size)
        step = half
        amp *= roughness
    return h


def fractal_heightmap(seed: int, n: int = 512, top: float = 300.0) -> np.ndarray:
    """Seeded n x n fp32 heightmap with values in [0, top] metres."""
    rng = np.random.default_rng(seed)
    h = diamond_square(rng, n_pow=int(np.ceil(np.log2(n))))[:n, :n]
    lo, hi = h.min(), h.max()
    return ((h - lo) / (hi - lo) * top).astype(np.float32)


def _cell_max(hm: np.ndarray, box, x: float, y: float) -> float:
    """Highest heightmap node of the grid cell containing (x, y) (input placement only)."""
    ny, nx = hm.shape
    fx = (x - box[0]) / (box[3] - box[0]) * (nx - 1)
    fy = (y - box[1]) / (box[4] - box[1]) * (ny - 1)
    ix = min(max(int(np.floor(fx)), 0), nx - 2)
    iy = min(max(int(np.floor(fy)), 0), ny - 2)
    return float(hm[iy:iy + 2, ix:ix + 2].max())


# ---------------------------------------------------------------------------
# plans


def sample_polyline(points: np.ndarray, speed: float, dt: float) -> np.ndarray:
    """Points every ``speed*dt`` metres of arc length along a polyline, ending at its end."""
    seg = np.diff(points, axis=0)
    seg_len = np.sqrt((seg ** 2).sum(axis=1))
    cum = np.concatenate([[0.0], np.cumsum(seg_len)])
    total = cum[-1]
    step = speed * dt
    n_full = int(np.floor(total / step))
    s = np.arange(n_full + 1) * step
    if total - s[-1] > 1e-9:
        s = np.concatenate([s, [total]])
    idx = np.clip(np.searchsorted(cum, s, side="right") - 1, 0, len(seg) - 1)
    frac = np.where(seg_len[idx] > 0, (s - cum[idx]) / np.maximum(seg_len[idx], 1e-300), 0.0)
    out = points[idx] + seg[idx] * frac[:, None]
    return out.astype(np.float32)


def _uniform_point(rng, box, zlo, zhi):
    return np.array([rng.uniform(box[0], box[3]), rng.uniform(box[1], box[4]), rng.uniform(zlo, zhi)])


def straight_plans(rng, box, n, zlo, zhi, vlo, vhi, tlo, thi, dt):
    plans = []
    for _ in range(n):
        o = _uniform_point(rng, box, zlo, zhi)
        d = _uniform_point(rng, box, zlo, zhi)
        v = rng.uniform(vlo, vhi)
        t0 = int(rng.integers(tlo, thi + 1))
        plans.append(Plan(t0, sample_polyline(np.stack([o, d]), v, dt)))
    return plans


def multileg_plans(rng, box, n, hm, legs=(3, 6), leg_len=(3000.0, 9000.0), zspan=(60.0, 600.0),
                   vlo=20.0, vhi=40.0, tlo=0, thi=1800, dt=1.0):
    plans = []
    for _ in range(n):
        k = int(rng.integers(legs[0], legs[1] + 1))
        pts = []
        x, y = rng.uniform(box[0], box[3]), rng.uniform(box[1], box[4])
        for i in range(k + 1):
            if i > 0:
                ang = rng.uniform(0.0, 2.0 * np.pi)
                L = rng.uniform(*leg_len)
                x = x + L * np.cos(ang)
                y = y + L * np.sin(ang)
                # reflect into the box
                if x < box[0]: x = 2 * box[0] - x
                if x > box[3]: x = 2 * box[3] - x
                if y < box[1]: y = 2 * box[1] - y
                if y > box[4]: y = 2 * box[4] - y
                x = min(max(x, box[0]), box[3]); y = min(max(y, box[1]), box[4])
            base = _cell_max(hm, box, x, y) if hm is not None else box[2]
            z = min(base + rng.uniform(*zspan), box[5] - 1.0)
            pts.append((x, y, z))
        v = rng.uniform(vlo, vhi)
        t0 = int(rng.integers(tlo, thi + 1))
        plans.append(Plan(t0, sample_polyline(np.array(pts, dtype=np.float64), v, dt)))
    return plans


def make_requests(rng, box, n, hm=None, zlo=50.0, zhi=450.0, zspan=(60.0, 500.0), vlo=20.0, vhi=40.0,
                  tlo=0, thi=600, horizon=1200, horizon_range=None, reach_frac=None, id0=1):
    req = np.zeros(n, dtype=REQUEST_DTYPE)
    for i in range(n):
        o = _uniform_point(rng, box, zlo, zhi)
        v = rng.uniform(vlo, vhi)
        H = int(rng.integers(horizon_range[0], horizon_range[1] + 1)) if horizon_range else horizon
        if reach_frac is not None:
            ang = rng.uniform(0.0, 2.0 * np.pi)
            L = reach_frac * v * H
            g = np.array([o[0] + L * np.cos(ang), o[1] + L * np.sin(ang), 0.0])
            g[0] = min(max(g[0], box[0]), box[3])
            g[1] = min(max(g[1], box[1]), box[4])
        else:
            g = _uniform_point(rng, box, zlo, zhi)
        if hm is not None:
            o[2] = min(_cell_max(hm, box, o[0], o[1]) + rng.uniform(*zspan), box[5] - 1.0)
            g[2] = min(_cell_max(hm, box, g[0], g[1]) + rng.uniform(*zspan), box[5] - 1.0)
        elif reach_frac is not None:
            g[2] = rng.uniform(zlo, zhi)
        req[i] = (id0 + i, o[0], o[1], o[2], g[0], g[1], g[2], v, int(rng.integers(tlo, thi + 1)), H)
    return req


# ---------------------------------------------------------------------------
# named workloads (shapes of the paper's FCFS experiment, Sec. V-VI)


def c1_plain_small(seed: int = 101) -> Scenario:
    """10 km x 10 km x 500 m, 200 straight known plans, 50 requests, 15 actions."""
    rng = np.random.default_rng(seed)
    box = (0.0, 0.0, 0.0, 10000.0, 10000.0, 500.0)
    plans = straight_plans(rng, box, 200, 50.0, 450.0, 20.0, 40.0, 0, 600, 1.0)
    reqs = make_requests(rng, box, 50, zlo=50.0, zhi=450.0, tlo=0, thi=600, horizon=1200)
    return Scenario("c1_plain_10km_200plans_50req_A15", box, 1.0, 0.99, action_grid((-2.0, 0.0, 2.0)),
                    (150.0, 30.0), plans, reqs, n_slices_window=2048, max_slots=512)


def e1_fine(seed: int = 106, n_plans: int = 60, n_requests: int = 12, lookahead_W: int = 10) -> Scenario:
    """The paper's own fidelity (Sec. IV "Forward project": W = 10 sub-steps of dt = 0.1 s):
    a 4 km x 4 km x 500 m box, straight known plans sampled every 0.1 s and departing within
    the first minute, and requests of up to 300 s that cross their paths; 15 actions. The
    lookahead window is a planning option (meta["lookahead_W"])."""
    rng = np.random.default_rng(seed)
    box = (0.0, 0.0, 0.0, 4000.0, 4000.0, 500.0)
    dt = 0.1
    plans = straight_plans(rng, box, n_plans, 100.0, 400.0, 20.0, 40.0, 0, 600, dt)
    reqs = make_requests(rng, box, n_requests, zlo=100.0, zhi=400.0, tlo=0, thi=600, horizon=3000)
    return Scenario(f"e1_fine_4km_{n_plans}plans_{n_requests}req_A15_dt0.1_W{lookahead_W}", box, dt, 0.99,
                    action_grid((-2.0, 0.0, 2.0)), (150.0, 30.0), plans, reqs, n_slices_window=4096,
                    max_slots=n_plans + n_requests + 32, meta={"lookahead_W": lookahead_W})


def c2_plain_scale(seed: int = 102, n_plans: int = 3000, n_requests: int = 1000) -> Scenario:
    """30 km x 30 km x 1 km with a 512^2 fractal heightmap (0-300 m, 60 m clearance),
    multi-leg known plans, FCFS requests with 25 actions and horizons up to 1800 steps."""
    hm = fractal_heightmap(seed)
    rng = np.random.default_rng(seed + 1000)
    box = (0.0, 0.0, 0.0, 30000.0, 30000.0, 1000.0)
    plans = multileg_plans(rng, box, n_plans, hm, tlo=0, thi=1800)
    reqs = make_requests(rng, box, n_requests, hm=hm, zspan=(60.0, 500.0), tlo=0, thi=1800, horizon=1800)
    return Scenario(f"c2_plain_30km_{n_plans}plans_{n_requests}req_A25", box, 1.0, 0.99,
                    action_grid((-4.0, -2.0, 0.0, 2.0, 4.0)), (150.0, 30.0), plans, reqs,
                    heightmap=hm, clearance=60.0, n_slices_window=4096,
                    max_slots=n_plans + n_requests + 128)


def c3_batched(seed: int = 103, n_plans: int = 20000, n_requests: int = 1024) -> Scenario:
    """C2's airspace with 20k known plans; requests with horizons U[60,1800] whose
    destination lies 0.8*v*H from the origin (clipped to the box)."""
    hm = fractal_heightmap(102)
    rng = np.random.default_rng(seed + 1000)
    box = (0.0, 0.0, 0.0, 30000.0, 30000.0, 1000.0)
    plans = multileg_plans(rng, box, n_plans, hm, tlo=0, thi=1800)
    reqs = make_requests(rng, box, n_requests, hm=hm, zspan=(60.0, 500.0), tlo=0, thi=1800,
                         horizon_range=(60, 1800), reach_frac=0.8)
    return Scenario(f"c3_batched_30km_{n_plans}plans_{n_requests}req_A25", box, 1.0, 0.99,
                    action_grid((-4.0, -2.0, 0.0, 2.0, 4.0)), (150.0, 30.0), plans, reqs,
                    heightmap=hm, clearance=60.0, n_slices_window=4096,
                    max_slots=n_plans + n_requests + 128)


def crowded_batch(seed: int = 104, n_plans: int = 200, n_requests: int = 48, spread_m: float = 1500.0,
                  depart_window: int = 30) -> Scenario:
    """C1's airspace and plan mix, with requests that leave one small region within a
    short window towards goals all around it, so that their paths cross while they fly
    (a stress case for speculative batching: many requests influence one another)."""
    rng = np.random.default_rng(seed)
    box = (0.0, 0.0, 0.0, 10000.0, 10000.0, 500.0)
    plans = straight_plans(rng, box, n_plans, 50.0, 450.0, 20.0, 40.0, 0, 600, 1.0)
    req = np.zeros(n_requests, dtype=REQUEST_DTYPE)
    cx, cy = 5000.0, 5000.0
    for i in range(n_requests):
        r, a = spread_m * np.sqrt(rng.uniform()), rng.uniform(0.0, 2.0 * np.pi)
        ox, oy = cx + r * np.cos(a), cy + r * np.sin(a)
        b, L = rng.uniform(0.0, 2.0 * np.pi), rng.uniform(3000.0, 4500.0)
        gx, gy = cx + L * np.cos(b), cy + L * np.sin(b)
        req[i] = (1 + i, ox, oy, rng.uniform(150.0, 350.0), gx, gy, rng.uniform(150.0, 350.0),
                  rng.uniform(20.0, 40.0), int(rng.integers(0, depart_window + 1)), 900)
    return Scenario(f"crowded_10km_{n_plans}plans_{n_requests}req_A15", box, 1.0, 0.99,
                    action_grid((-2.0, 0.0, 2.0)), (150.0, 30.0), plans, req, n_slices_window=2048,
                    max_slots=n_plans + n_requests + 64)


def c4_serving(seed: int = 104, n_plans: int = 100000) -> Scenario:
    """Serving workload: C2's airspace and terrain (30 km x 30 km x 1 km) with `n_plans` known
    plans in a sliding window of 4096 steps, room for 100k active plans plus the requests.
    Known plans are 1-2 legs of 2-6 km departing U[0, 3000] s, about 200 s of flight each, so
    some 6-7k of them are in the air at a time (the 20k-plan workload's density). Serving
    starts its simulated clock at step meta["sim_start"] (plans that ended before it can be
    expired at once); `serving_requests` makes the arrivals, `sweep_requests` a batch."""
    hm = fractal_heightmap(102)
    rng = np.random.default_rng(seed + 1000)
    box = (0.0, 0.0, 0.0, 30000.0, 30000.0, 1000.0)
    plans = multileg_plans(rng, box, n_plans, hm, legs=(1, 2), leg_len=(2000.0, 6000.0), tlo=0, thi=3000)
    return Scenario(f"c4_serving_30km_{n_plans}plans_A25", box, 1.0, 0.99,
                    action_grid((-4.0, -2.0, 0.0, 2.0, 4.0)), (150.0, 30.0), plans,
                    np.zeros(0, dtype=REQUEST_DTYPE), heightmap=hm, clearance=60.0, n_slices_window=4096,
                    max_slots=n_plans + 16384, meta={"max_active_plans": 100000, "sim_start": 600})


def sweep_requests(sc: Scenario, n: int, seed: int, tlo: int = 600, thi: int = 2000) -> np.ndarray:
    """A batch of FCFS requests shaped like the 20k-plan workload's (horizons U[60, 1800],
    destination 0.8 v H from the origin), departing U[tlo, thi]."""
    rng = np.random.default_rng(seed)
    return make_requests(rng, sc.box, n, hm=sc.heightmap, zspan=(60.0, 500.0), tlo=tlo, thi=thi,
                         horizon_range=(60, 1800), reach_frac=0.8)


def poisson_arrivals(seed: int, rate_per_s: float, duration_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate over [0, duration)."""
    rng = np.random.default_rng(seed)
    n = max(1, int(rate_per_s * duration_s * 1.5) + 16)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    return t[t < duration_s]


def serving_requests(sc: Scenario, arrival_s: np.ndarray, seed: int, time_scale: float,
                     lead_s=(120.0, 600.0), horizon_range=(60, 1200), reach_frac=0.5,
                     sim_start: int = 0) -> np.ndarray:
    """One request per arrival: it departs `lead` simulated seconds after its arrival on the
    simulated clock (sim_start + arrival x time_scale), towards a destination reach_frac v H
    away."""
    rng = np.random.default_rng(seed)
    req = make_requests(rng, sc.box, len(arrival_s), hm=sc.heightmap, zspan=(60.0, 500.0), tlo=0, thi=0,
                        horizon_range=horizon_range, reach_frac=reach_frac)
    lead = rng.uniform(*lead_s, size=len(arrival_s))
    req["depart"] = sim_start + np.floor((arrival_s * time_scale + lead) / sc.dt).astype(np.int64)
    return req


def sort_plans_by_departure(plans: List[Plan]) -> List[Plan]:
    """Stable order by departure step (slot allocation then groups plans in time)."""
    order = sorted(range(len(plans)), key=lambda i: (plans[i].t0, i))
    return [plans[i] for i in order]
