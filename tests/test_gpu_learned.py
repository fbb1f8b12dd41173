"""The learned proposal on the GPU against its FP64 oracle (oracle/learned.py).

- features: the rows the collector writes for a FastMDP rollout equal the oracle's
  features of the same states (bf16 storage; a sample that sits on a sector boundary may
  fall on either side, so a few rows may differ in one sector);
- gradient: the GPU's forward and backward kernels (bf16 tensor-core GEMMs, fp32
  accumulation) against the oracle's exact FP64 gradient of the same bf16 network;
- training: the loss falls, and the trained network's proposals are accepted far more
  often than an untrained one's (what the network gains over the method without it);
- scheduling: learned FCFS gives the same results whatever the batch size (one request
  per batch is the sequential rule), every accepted proposal is admitted, and the
  accepted proposals replace FastMDP rollouts.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import ADMITTED  # noqa: E402
from oracle import learned as OL  # noqa: E402
from paper_2008_03518_gb300 import scenarios as S  # noqa: E402
from paper_2008_03518_gb300.fmdp import MLP_PARAMS, Scheduler  # noqa: E402

from test_gpu_batch import same_results  # noqa: E402


def bf16(x):
    """Round float32 values to the nearest bfloat16 (ties to even), kept as float32."""
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    a = (a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000
    return a.astype(np.uint32).view(np.float32)


def plan_samples(sc, t):
    """Every known plan's sample at step t and at t + 1 (NaN where it has none)."""
    p1, p2 = [], []
    for pl in sc.plans:
        j = t - pl.t0
        if 0 <= j < len(pl.xyz):
            p1.append(pl.xyz[j])
            p2.append(pl.xyz[j + 1] if j + 1 < len(pl.xyz) else np.full(3, np.nan, np.float32))
    return np.array(p1, dtype=np.float64).reshape(-1, 3), np.array(p2, dtype=np.float64).reshape(-1, 3)


def test_collected_features_match_the_oracle():
    sc = S.c1_plain_small()
    reqs = sc.requests[:3]
    with Scheduler.from_scenario(sc) as s:
        rows = s.learned_collect(reqs)
        X, y = s.learned_rows(rows)
        traces = [s.rollout_trace(r) for r in reqs]
    assert rows == sum(t["n_points"] - 1 for t in traces) and rows > 100
    o = 0
    bad = 0
    worst = 0.0
    for r, t in zip(reqs, traces):
        c0, s0 = r["gx"] - r["ox"], r["gy"] - r["oy"]
        L = np.hypot(c0, s0)
        c0, s0 = c0 / L, s0 / L
        for k in range(t["n_points"] - 1):
            a = np.pi / 12.0 * t["headings"][k]
            hc, hs = c0 * np.cos(a) - s0 * np.sin(a), s0 * np.cos(a) + c0 * np.sin(a)
            p1, p2 = plan_samples(sc, int(r["depart"]) + k + 1)
            want = OL.features(t["xyz"][k].astype(np.float64), hc, hs, float(r["speed"]),
                               (r["gx"], r["gy"], r["gz"]), sc.box, p1, p2, dt=sc.dt)
            assert y[o + k] == t["actions"][k]
            err = np.abs(X[o + k] - want)
            tol = 8e-3 * np.abs(want) + 2e-3
            if np.any(err > tol):
                bad += 1
                worst = max(worst, float(np.max(err - tol)))
        o += t["n_points"] - 1
    assert bad <= max(2, rows // 100), (bad, rows, worst)


def test_collect_writes_every_row_of_a_rollout_longer_than_2047_steps():
    """A rollout at dt = 0.1 s that runs well past 2047 steps: the collector writes exactly
    the n_points - 1 rows the host counts for it, each row the oracle's features of that
    state and its label the action FastMDP took there."""
    sc = S.e1_fine(lookahead_W=1)
    req = np.zeros(1, dtype=S.REQUEST_DTYPE)
    req[0] = (1, 150.0, 150.0, 250.0, 3850.0, 3850.0, 250.0, 20.0, 0, 4000)
    with Scheduler.from_scenario(sc) as s:
        rows = s.learned_collect(req)
        X, y = s.learned_rows(rows + 16)
        t = s.rollout_trace(req[0])
    n = t["n_points"] - 1
    assert n > 2047 + 300 and rows == n and len(X) == n, (n, rows, len(X))
    np.testing.assert_array_equal(y, t["actions"][:n])
    r = req[0]
    c0, s0 = r["gx"] - r["ox"], r["gy"] - r["oy"]
    L = np.hypot(c0, s0)
    c0, s0 = c0 / L, s0 / L
    bad = []
    with_intruders = 0
    for k in range(n):
        a = np.pi / 12.0 * t["headings"][k]
        hc, hs = c0 * np.cos(a) - s0 * np.sin(a), s0 * np.cos(a) + c0 * np.sin(a)
        p1, p2 = plan_samples(sc, int(r["depart"]) + k + 1)
        want = OL.features(t["xyz"][k].astype(np.float64), hc, hs, float(r["speed"]),
                           (r["gx"], r["gy"], r["gz"]), sc.box, p1, p2, dt=sc.dt)
        with_intruders += bool(np.any(want[OL.N_OWN:] != 0.0))
        if np.any(np.abs(X[k] - want) > 8e-3 * np.abs(want) + 2e-3):
            bad.append(k)
    # a sample on a sector boundary may fall on either side: a few rows, never a run of them
    assert len(bad) <= max(2, n // 100), (len(bad), n, bad[:10])
    assert with_intruders > 20  # the rows past the old limit are not all own-state only


def test_gradient_matches_the_oracle():
    """GPU loss and gradient against the oracle's bf16 network (the same rounding points:
    bf16 weights, hidden activations and matrix-product operands, fp32 accumulation), and
    against the exact FP64 gradient within what that rounding costs on this batch."""
    sc = S.c1_plain_small()
    rng = np.random.default_rng(5)
    with Scheduler.from_scenario(sc, add_plans=False) as s:
        s.learned_init(seed=11)
        p = s.learned_get_params()
        X = bf16(rng.normal(0.0, 0.7, size=(96, 128)))
        y = rng.integers(0, len(sc.actions), size=96).astype(np.uint8)
        loss, g = s.learned_loss_grad(X, y)
    q = p.astype(np.float64).copy()
    for (o_w, n_w) in _weight_blocks():
        q[o_w:o_w + n_w] = bf16(p[o_w:o_w + n_w])
    A = len(sc.actions)
    r_loss, r_g = OL.loss_and_grad(q, X.astype(np.float64), y, n_valid=A, round_fn=OL.bf16)
    e_loss, e_g = OL.loss_and_grad(q, X.astype(np.float64), y, n_valid=A)
    assert abs(loss - r_loss) <= 1e-4 * r_loss and abs(loss - e_loss) <= 1e-2 * e_loss
    for (o_w, n_w), (o_b, n_b) in zip(_weight_blocks(), _bias_blocks()):
        for o, n in ((o_w, n_w), (o_b, n_b)):
            sl = slice(o, o + n)
            # Element by element against the bf16 oracle. Both sides round at the same
            # points; they differ only where the GPU's fp32 accumulation (another order than
            # the oracle's FP64 sums) lands an activation or an output gradient on the other
            # side of a bf16 rounding boundary, which moves that value by one bf16 ulp
            # (2^-8 relative) and the gradient elements it feeds by at most that share.
            # rtol 2e-2 covers such an ulp on an element it dominates; the absolute floor
            # (2e-3 of the block's largest element) covers elements near zero. A wrong sign,
            # a transposed block or a swapped index moves elements by 100 % or more.
            scale = float(np.abs(r_g[sl]).max())
            np.testing.assert_allclose(g[sl], r_g[sl], rtol=2e-2, atol=2e-3 * scale,
                                       err_msg=f"gradient block at offset {o}")
            # the signs of the clearly non-zero elements agree with the oracle's
            big = np.abs(r_g[sl]) > 0.05 * scale
            assert np.array_equal(np.sign(g[sl][big]), np.sign(r_g[sl][big])), o
            # and against the exact FP64 gradient, within what the bf16 rounding costs
            rel_e = np.linalg.norm(g[sl] - e_g[sl]) / max(np.linalg.norm(e_g[sl]), 1e-12)
            bound = np.linalg.norm(r_g[sl] - e_g[sl]) / max(np.linalg.norm(e_g[sl]), 1e-12)
            assert rel_e < 1.5 * bound + 1e-2, (o, rel_e, bound)
    assert g.shape == (MLP_PARAMS,)


def _weight_blocks():
    out, o = [], 0
    for a, b in zip(OL.DIMS[:-1], OL.DIMS[1:]):
        out.append((o, a * b))
        o += a * b + b
    return out


def _bias_blocks():
    out, o = [], 0
    for a, b in zip(OL.DIMS[:-1], OL.DIMS[1:]):
        out.append((o + a * b, b))
        o += a * b + b
    return out


@pytest.fixture(scope="module")
def trained():
    """A network trained on FastMDP rollouts of C1-shaped traffic."""
    sc = S.c1_plain_small()
    rng = np.random.default_rng(9)
    train_reqs = S.make_requests(rng, sc.box, 120, zlo=50.0, zhi=450.0, tlo=0, thi=600, horizon=1200, id0=1000)
    with Scheduler.from_scenario(sc) as s:
        rows = s.learned_collect(train_reqs)
        s.learned_init(seed=3)
        losses = s.learned_train(epochs=8, batch=256, lr=2e-3, seed=4)
        params = s.learned_get_params()
    return sc, params, losses, rows


def test_training_reduces_the_loss(trained):
    sc, params, losses, rows = trained
    assert rows > 20000
    assert losses[-1] < 0.7 * losses[0] and losses[-1] < 1.0, losses
    assert np.all(np.diff(losses) < 0.02), losses  # no epoch makes it clearly worse


def test_trained_proposals_beat_untrained_ones(trained):
    sc, params, _, _ = trained
    reqs = sc.requests
    with Scheduler.from_scenario(sc) as s:
        s.learned_init(seed=3)
        rep0, acc0, _, _ = s.learned_evaluate(reqs)
        s.learned_set_params(params)
        rep1, acc1, sp, sf = s.learned_evaluate(reqs)
    assert rep1["accepted"] >= max(5, 3 * rep0["accepted"]), (rep0, rep1)
    # accepted proposals are never more than 5 % longer than a FastMDP plan that reaches
    # the goal (max_gap covers those; an accepted proposal may also reach a goal that
    # FastMDP's own rollout does not)
    assert rep1["max_gap"] <= 0.05 + 1e-12 and rep1["mean_gap"] <= 0.05
    assert rep1["accepted"] <= rep1["proposals_captured"]


def test_learned_fcfs_is_batch_independent_and_replaces_rollouts(trained):
    sc, params, _, _ = trained
    out = []
    for bs in (1, 16):
        with Scheduler.from_scenario(sc, batch_size=bs) as s:
            s.learned_set_params(params)
            s.set_profiling(1)
            res, rep = s.schedule_learned(sc.requests)
            st = s.stats()
            out.append((res, rep, st))
    (r1, rep1, st1), (r2, rep2, st2) = out
    same_results(r1, r2)
    assert [x["source"] for x in r1] == [x["source"] for x in r2]
    assert rep1["accepted"] == rep2["accepted"] > 0
    assert all(x["verdict"] == ADMITTED for x in r1 if x["source"] == 1)
    with Scheduler.from_scenario(sc) as s:
        s.set_profiling(1)
        s.schedule_batch(sc.requests)
        plain_steps = s.stats()["rollout_steps"]
    assert st2["rollout_steps"] < plain_steps  # FastMDP ran only for the rejected proposals


def test_learned_fcfs_against_plain_fastmdp_on_the_same_requests(trained):
    """Learned FCFS (accepted proposal, else FastMDP) against plain FastMDP FCFS over the
    same requests and table: the proposals replace FastMDP rollout steps, every accepted
    proposal is admitted and costs at most 5 % more steps than FastMDP's own plan of that
    request (C5's gap bound), and both paths' wall times are measured and reported."""
    import time

    sc, params, _, _ = trained
    out = {}
    for label in ("plain", "learned"):
        with Scheduler.from_scenario(sc) as s:
            s.learned_set_params(params)
            s.set_profiling(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if label == "plain":
                res = s.schedule_batch(sc.requests)
            else:
                res, rep = s.schedule_learned(sc.requests)
            torch.cuda.synchronize()
            out[label] = (res, s.stats(), time.perf_counter() - t0)
    (rp, sp, wp), (rl, sl, wl) = out["plain"], out["learned"]
    assert wp > 0 and wl > 0
    print(f"plain FastMDP FCFS: {wp * 1e3:.1f} ms, {sp['rollout_steps']} rollout steps; "
          f"learned FCFS: {wl * 1e3:.1f} ms, {sl['rollout_steps']} FastMDP rollout steps")
    acc = [i for i, r in enumerate(rl) if r["source"] == 1]
    assert acc and sl["rollout_steps"] < sp["rollout_steps"]
    assert all(rl[i]["verdict"] == ADMITTED for i in acc)
    # the first accepted proposal met the same table as plain FastMDP (nothing admitted
    # differently before it): its cost is within 5 % of FastMDP's plan
    first = acc[0]
    if all(rl[i]["plan_id"] == rp[i]["plan_id"] and rl[i]["verdict"] == rp[i]["verdict"] for i in range(first)):
        assert rl[first]["n_points"] - 1 <= 1.05 * (rp[first]["n_points"] - 1) + 1e-9
