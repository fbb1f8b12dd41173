"""Helpers shared by the GPU parity tests: the CUDA scheduler is compared with the FP64
oracle element by element on the same seeded inputs.

Bars (from the method's statement of parity):
  * per-action Q within 1e-5 of the action's term scale max(goal term, penalty + deck);
  * identical action sequence except at near-ties (top-2 gap < 1e-4 of the scale), where
    the oracle follows the GPU's choice (lock-step / teacher forcing);
  * bit-identical trajectories (the FP64 state advance is exact on both sides) and
    bit-identical admit / reject verdicts and first-conflict indices.
"""
import numpy as np

from oracle import ADMITTED, REJ_CONFLICT, REJ_TERRAIN, Oracle

Q_REL = 1e-5
SEP_REL = 1e-5


def oracle_for(sc, **kw):
    return Oracle.from_scenario(sc, **kw)


def check_q(gq, oq, oscale, where=""):
    """GPU fp64 action values vs oracle values at the same states."""
    assert gq.shape == oq.shape, (gq.shape, oq.shape, where)
    inv_g, inv_o = ~np.isfinite(gq), ~np.isfinite(oq)
    np.testing.assert_array_equal(inv_g, inv_o, err_msg=f"validity differs {where}")
    ok = np.isfinite(oq)
    err = np.abs(gq[ok] - oq[ok])
    tol = Q_REL * oscale[ok] + 1e-300
    bad = err > tol
    if bad.any():
        i = np.argmax(err / tol)
        raise AssertionError(f"Q mismatch {where}: max err/tol={float((err / tol)[i]):.3g} "
                             f"gpu={gq[ok][i]!r} oracle={oq[ok][i]!r} scale={oscale[ok][i]!r}")


def follow_and_check(o, req, g, check_sep=True):
    """Runs the oracle teacher-forced on the GPU's actions, checks the trajectory bit for
    bit and returns the oracle's verdict for it (before admission)."""
    acts = np.asarray(g["actions"], dtype=np.int32)
    d = o.rollout(req, follow=acts)
    assert d["mismatch_step"] == -1, f"GPU action at step {d['mismatch_step']} is not a near-tie of the oracle's"
    assert d["n_points"] == g["n_points"], (d["n_points"], g["n_points"])
    np.testing.assert_array_equal(d["xyz"], g["xyz"])
    chk = o.sep_check(_depart(req), d["xyz"])
    if d["verdict"] >= 0:  # rollout failed: horizon or no valid action
        verdict = d["verdict"]
    elif chk["first_conflict"] >= 0:
        verdict = REJ_CONFLICT
    elif chk["first_terrain"] >= 0:
        verdict = REJ_TERRAIN
    else:
        verdict = ADMITTED
    if check_sep:
        assert g["first_conflict_step"] == chk["first_conflict"]
        assert g["first_terrain_step"] == chk["first_terrain"]
        for k in ("min_sep_h", "min_sep_v"):
            a, b = g[k], chk[k]
            if np.isfinite(b):
                assert abs(a - b) <= SEP_REL * max(b, 1.0), (k, a, b)
            else:
                assert not np.isfinite(a), (k, a, b)
    return verdict, d


def _names(req):
    return req.dtype.names if hasattr(req, "dtype") else tuple(req.keys())


def _depart(req):
    return int(req["depart"]) if "depart" in _names(req) else int(req["depart_step"])


def fcfs_parity(gpu, o, reqs, trace_q=False, gpu_results=None):
    """FCFS over reqs on both sides; the oracle follows the GPU at near-ties and stores
    what it admits. Returns (verdicts, followed near-ties, steps)."""
    verdicts, followed, steps = [], 0, 0
    for i, r in enumerate(reqs):
        if trace_q:
            t = gpu.rollout_trace(r)
            d = o.rollout(r, follow=np.asarray(t["actions"], dtype=np.int32), trace=True)
            assert d["mismatch_step"] == -1, f"request {i}: trace action not a near-tie at {d['mismatch_step']}"
            np.testing.assert_array_equal(d["xyz"], t["xyz"])
            np.testing.assert_array_equal(d["states"], t["states"])
            check_q(t["q"], d["q"], d["scale"], where=f"request {i}")
        g = gpu_results[i] if gpu_results is not None else gpu.schedule(r)
        v, d = follow_and_check(o, r, g)
        assert g["verdict"] == v, f"request {i}: gpu verdict {g['verdict']} oracle {v}"
        if v == ADMITTED:
            o.add_plan(_depart(r), d["xyz"])
        followed += d["followed_ties"]
        steps += max(int(g["n_points"]) - 1, 0)
        verdicts.append(v)
    return verdicts, followed, steps
