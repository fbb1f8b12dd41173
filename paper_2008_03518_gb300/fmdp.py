"""ctypes binding of libfmdp.so: the same entry points as include/fmdp.h.

Argument marshalling only: every step of planning runs in the library's CUDA kernels.
There is no CPU fallback; constructing a Scheduler without the compiled library or
without a CUDA device raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

ADMITTED, REJ_CONFLICT, REJ_TERRAIN, REJ_HORIZON, REJ_NO_ACTION = range(5)
STATUS_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_TIMEOUT", -5: "ERR_FULL",
                -6: "ERR_RANGE", -7: "ERR_NOTFOUND", -8: "ERR_IO"}


def append_jsonl(path, record):
    """Appends one metrics record as a JSON line (numpy scalars and arrays as plain numbers
    and lists) to the file at path."""
    import json

    def plain(v):
        if isinstance(v, dict):
            return {str(k): plain(x) for k, x in v.items()}
        if isinstance(v, (list, tuple)):
            return [plain(x) for x in v]
        if isinstance(v, np.ndarray):
            return v.tolist()
        if isinstance(v, np.generic):
            return v.item()
        return v

    with open(path, "a", encoding="utf-8") as f:
        f.write(json.dumps(plain(record), sort_keys=True) + "\n")


class FmdpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)


class Airspace(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
                ("x1", ctypes.c_double), ("y1", ctypes.c_double), ("z1", ctypes.c_double),
                ("dt", ctypes.c_double), ("n_slices_window", ctypes.c_int32), ("max_slots", ctypes.c_int32),
                ("heightmap", _fp), ("hm_nx", ctypes.c_int32), ("hm_ny", ctypes.c_int32),
                ("clearance_m", ctypes.c_double), ("deck_value", ctypes.c_double),
                ("static_wells", _dp), ("n_static_wells", ctypes.c_int32)]


class Action(ctypes.Structure):
    _fields_ = [("dpsi_deg", ctypes.c_double), ("climb_mps", ctypes.c_double)]


class Sep(ctypes.Structure):
    _fields_ = [("horiz_m", ctypes.c_double), ("vert_m", ctypes.c_double)]


class Well(ctypes.Structure):
    _fields_ = [("tau_s", ctypes.c_double), ("radius_m", ctypes.c_double), ("magnitude", ctypes.c_double),
                ("gamma", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("combine", ctypes.c_int32), ("wells", ctypes.POINTER(Well)), ("n_wells", ctypes.c_int32),
                ("goal_reward", ctypes.c_double), ("lookahead_W", ctypes.c_int32),
                ("cluster_size", ctypes.c_int32), ("threads_per_cta", ctypes.c_int32), ("batch_size", ctypes.c_int32),
                ("full_scan", ctypes.c_int32), ("index_vmax_mps", ctypes.c_double), ("index_cell_m", ctypes.c_double),
                ("index_stage_items", ctypes.c_int32), ("batch_mode", ctypes.c_int32),
                ("pipe_rebuild_items", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("req_id", ctypes.c_uint64), ("ox", ctypes.c_double), ("oy", ctypes.c_double),
                ("oz", ctypes.c_double), ("gx", ctypes.c_double), ("gy", ctypes.c_double), ("gz", ctypes.c_double),
                ("speed_mps", ctypes.c_double), ("depart_step", ctypes.c_int64), ("horizon", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("verdict", ctypes.c_int32), ("n_points", ctypes.c_int32), ("plan_id", ctypes.c_uint64),
                ("first_conflict_step", ctypes.c_int32), ("first_terrain_step", ctypes.c_int32),
                ("min_sep_h", ctypes.c_double), ("min_sep_v", ctypes.c_double), ("near_ties", ctypes.c_int32),
                ("replanned", ctypes.c_int32), ("source", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("xyz", _fp), ("actions", ctypes.POINTER(ctypes.c_uint8))]


class SepReport(ctypes.Structure):
    _fields_ = [("first_conflict_step", ctypes.c_int32), ("first_terrain_step", ctypes.c_int32),
                ("conflicts", ctypes.c_int64), ("min_sep_h", ctypes.c_double), ("min_sep_v", ctypes.c_double)]


MLP_PARAMS = 236825


class LearnedReport(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("accepted", ctypes.c_int32), ("proposals_captured", ctypes.c_int32),
                ("fastmdp_captured", ctypes.c_int32), ("mean_gap", ctypes.c_double), ("max_gap", ctypes.c_double),
                ("proposal_steps", ctypes.c_int64), ("fastmdp_steps", ctypes.c_int64),
                ("proposal_ms", ctypes.c_double), ("fastmdp_ms", ctypes.c_double)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("n_actions", ctypes.c_int32), ("combine", ctypes.c_int32), ("plans_bucket", ctypes.c_int32),
                ("wave_bucket", ctypes.c_int32), ("threads_per_cta", ctypes.c_int32),
                ("index_stage_items", ctypes.c_int32), ("ms", ctypes.c_double)]


class TuneReport(ctypes.Structure):
    _fields_ = [("chosen", TuneEntry), ("candidates", ctypes.c_int32), ("entries", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("from_cache", ctypes.c_int32), ("sample", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("default_ms", ctypes.c_double)]


def _entry_dict(e):
    return {k: getattr(e, k) for k, _ in TuneEntry._fields_}


class ServeOptions(ctypes.Structure):
    _fields_ = [("time_scale", ctypes.c_double), ("sim_start_step", ctypes.c_int64), ("sim_start_set", ctypes.c_int32),
                ("max_in_flight", ctypes.c_int32), ("max_active_plans", ctypes.c_int32),
                ("expire_quantum", ctypes.c_int32)]


class ServeReport(ctypes.Structure):
    _fields_ = [("wall_s", ctypes.c_double), ("throughput_rps", ctypes.c_double),
                ("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double),
                ("latency_mean_ms", ctypes.c_double), ("latency_max_ms", ctypes.c_double),
                ("waves", ctypes.c_int64), ("rollouts", ctypes.c_int64), ("replans", ctypes.c_int64),
                ("expiries", ctypes.c_int64), ("plans_expired", ctypes.c_int64), ("final_t_base", ctypes.c_int64),
                ("admitted", ctypes.c_int32), ("rejected", ctypes.c_int32), ("max_in_flight_seen", ctypes.c_int32),
                ("deferred_for_memory", ctypes.c_int32), ("pipelined", ctypes.c_int32),
                ("persistent_ctas", ctypes.c_int32), ("drains", ctypes.c_int64), ("rollout_occupancy", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("rollout_launches", ctypes.c_int64), ("sepcheck_launches", ctypes.c_int64),
                ("admit_launches", ctypes.c_int64), ("rollout_ms", ctypes.c_double),
                ("sepcheck_ms", ctypes.c_double), ("admit_ms", ctypes.c_double),
                ("rollout_steps", ctypes.c_int64), ("slots_scanned", ctypes.c_int64),
                ("sep_pairs", ctypes.c_int64), ("cluster_size", ctypes.c_int32),
                ("threads_per_cta", ctypes.c_int32), ("slots_per_cta", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("phase_cycles", ctypes.c_int64 * 6),
                ("batch_waves", ctypes.c_int64), ("batch_rollouts", ctypes.c_int64), ("batch_replans", ctypes.c_int64),
                ("influence_launches", ctypes.c_int64), ("influence_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("items_scanned", ctypes.c_int64),
                ("pipe_drains", ctypes.c_int64), ("pipe_cta_s", ctypes.c_double), ("pipe_slot_s", ctypes.c_double),
                ("pipe_ctas", ctypes.c_int32), ("pipe_resident", ctypes.c_int32),
                ("pipe_resumes", ctypes.c_int64), ("pipe_rechecks", ctypes.c_int64),
                ("qe_items", ctypes.c_int64), ("qe_near", ctypes.c_int64), ("qe_wells", ctypes.c_int64),
                ("pipe_head_n", ctypes.c_int64 * 5), ("pipe_head_s", ctypes.c_double * 5),
                ("pipe_publishes", ctypes.c_int64), ("pipe_withdrawals", ctypes.c_int64)]


class Peaks(ctypes.Structure):
    _fields_ = [("fp32_tflops", ctypes.c_double), ("mufu_rsqrt_tops", ctypes.c_double),
                ("mufu_ex2_tops", ctypes.c_double), ("sm_mhz", ctypes.c_double)]


# every exported symbol of include/fmdp.h
EXPORTS = ("fmdp_options_default", "fmdp_create", "fmdp_destroy", "fmdp_last_error", "fmdp_set_stream",
           "fmdp_add_plan", "fmdp_add_plans", "fmdp_schedule", "fmdp_schedule_many", "fmdp_schedule_batch",
           "fmdp_stage_requests", "fmdp_schedule_staged", "fmdp_fetch_staged", "fmdp_query_plans",
           "fmdp_serve", "fmdp_serve_options_default",
           "fmdp_learned_collect", "fmdp_learned_rows", "fmdp_learned_clear_rows", "fmdp_learned_init",
           "fmdp_learned_set_params", "fmdp_learned_get_params", "fmdp_learned_train", "fmdp_learned_loss_grad",
           "fmdp_learned_evaluate", "fmdp_schedule_learned",
           "fmdp_autotune", "fmdp_tune_cache_get", "fmdp_tune_cache_put", "fmdp_schedule_departures",
           "fmdp_schedule_departures_batch",
           "fmdp_schedule_cosim", "fmdp_selftest_wait_timeout",
           "fmdp_get_plan", "fmdp_save_plans", "fmdp_load_plans", "fmdp_expire", "fmdp_snapshot", "fmdp_restore", "fmdp_clear", "fmdp_rollout_trace",
           "fmdp_sep_check", "fmdp_sep_check_noalloc", "fmdp_set_profiling", "fmdp_get_stats",
           "fmdp_set_batch_mode", "fmdp_last_call_times", "fmdp_probe_peaks")

NOALLOC_MAX_POINTS = 16384  # FMDP_NOALLOC_MAX_POINTS

_lib = None


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Loads libfmdp.so (building it first if allowed). Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and _build.stale():
        _build.build()
    if not os.path.exists(_build.LIB_PATH):
        raise RuntimeError("libfmdp.so is not built; run paper_2008_03518_gb300.build.build()")
    L = ctypes.CDLL(_build.LIB_PATH)
    P, c = ctypes.POINTER, ctypes
    vp = c.c_void_p
    L.fmdp_options_default.argtypes = [P(Options)]
    L.fmdp_options_default.restype = None
    L.fmdp_create.argtypes = [P(Airspace), c.c_double, P(Action), c.c_int32, P(Sep), P(Options), P(vp)]
    L.fmdp_destroy.argtypes = [vp]
    L.fmdp_destroy.restype = None
    L.fmdp_last_error.argtypes = [vp]
    L.fmdp_last_error.restype = c.c_char_p
    L.fmdp_set_stream.argtypes = [vp, vp]
    L.fmdp_add_plan.argtypes = [vp, c.c_int64, _fp, c.c_int32, P(c.c_uint64)]
    L.fmdp_add_plans.argtypes = [vp, c.c_int32, P(c.c_int64), P(c.c_int32), _fp, P(c.c_uint64)]
    for name in ("fmdp_schedule_many", "fmdp_schedule_batch"):
        getattr(L, name).argtypes = [vp, P(Request), c.c_int32, P(Result)]
    L.fmdp_schedule.argtypes = [vp, P(Request), P(Result)]
    L.fmdp_stage_requests.argtypes = [vp, P(Request), c.c_int32]
    L.fmdp_schedule_staged.argtypes = [vp, c.c_int32, P(c.c_int32)]
    L.fmdp_learned_collect.argtypes = [vp, P(Request), c.c_int32, P(c.c_int32)]
    L.fmdp_learned_rows.argtypes = [vp, _fp, P(c.c_uint8), c.c_int32, P(c.c_int32)]
    L.fmdp_learned_clear_rows.argtypes = [vp]
    L.fmdp_learned_init.argtypes = [vp, c.c_uint64]
    L.fmdp_learned_set_params.argtypes = [vp, _fp, c.c_int32]
    L.fmdp_learned_get_params.argtypes = [vp, _fp, c.c_int32]
    L.fmdp_learned_train.argtypes = [vp, c.c_int32, c.c_int32, c.c_float, c.c_uint64, _fp]
    L.fmdp_learned_loss_grad.argtypes = [vp, _fp, P(c.c_uint8), c.c_int32, _fp, _fp]
    L.fmdp_learned_evaluate.argtypes = [vp, P(Request), c.c_int32, c.c_double, P(LearnedReport), P(c.c_int32),
                                        P(c.c_int32), P(c.c_int32)]
    L.fmdp_schedule_learned.argtypes = [vp, P(Request), c.c_int32, c.c_double, P(Result), P(LearnedReport)]
    L.fmdp_autotune.argtypes = [vp, P(Request), c.c_int32, c.c_int32, P(TuneReport)]
    L.fmdp_schedule_cosim.argtypes = [vp, P(Request), c.c_int32, P(Result)]
    L.fmdp_selftest_wait_timeout.argtypes = [vp, P(c.c_int32)]
    L.fmdp_schedule_departures.argtypes = [vp, P(Request), c.c_int32, P(c.c_int64), c.c_int32, P(Result),
                                           P(c.c_int32), P(c.c_int32)]
    L.fmdp_schedule_departures_batch.argtypes = L.fmdp_schedule_departures.argtypes
    L.fmdp_tune_cache_get.argtypes = [vp, P(TuneEntry), c.c_int32, P(c.c_int32)]
    L.fmdp_tune_cache_put.argtypes = [vp, P(TuneEntry), c.c_int32]
    L.fmdp_serve_options_default.argtypes = [P(ServeOptions)]
    L.fmdp_serve_options_default.restype = None
    L.fmdp_serve.argtypes = [vp, P(Request), P(c.c_double), c.c_int32, P(ServeOptions), P(Result), P(c.c_double),
                             P(ServeReport)]
    L.fmdp_fetch_staged.argtypes = [vp, P(Result), c.c_int32]
    L.fmdp_query_plans.argtypes = [vp, c.c_int64, c.c_int64, P(c.c_uint64), c.c_int32, P(c.c_int32)]
    L.fmdp_get_plan.argtypes = [vp, c.c_uint64, P(c.c_int64), _fp, c.c_int32, P(c.c_int32)]
    L.fmdp_save_plans.argtypes = [vp, c.c_char_p, P(c.c_int64)]
    L.fmdp_load_plans.argtypes = [vp, c.c_char_p, P(c.c_uint64), c.c_int64, P(c.c_int64)]
    L.fmdp_expire.argtypes = [vp, c.c_int64]
    for name in ("fmdp_snapshot", "fmdp_restore", "fmdp_clear"):
        getattr(L, name).argtypes = [vp]
    L.fmdp_rollout_trace.argtypes = [vp, P(Request), P(Result), _dp, _dp, P(c.c_int32), P(c.c_uint8)]
    L.fmdp_sep_check.argtypes = [vp, c.c_int64, _fp, c.c_int32, P(SepReport)]
    L.fmdp_sep_check_noalloc.argtypes = [vp, c.c_int64, _fp, c.c_int32, P(SepReport)]
    L.fmdp_set_profiling.argtypes = [vp, c.c_int32]
    L.fmdp_get_stats.argtypes = [vp, P(Stats)]
    L.fmdp_set_batch_mode.argtypes = [vp, c.c_int32]
    L.fmdp_last_call_times.argtypes = [vp, _dp, c.c_int32, P(c.c_int32)]
    L.fmdp_probe_peaks.argtypes = [vp, P(Peaks)]
    for name in EXPORTS:
        f = getattr(L, name)
        if f.restype is ctypes.c_int:  # default restype: all statuses are int32
            f.restype = c.c_int32
    _lib = L
    return L


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def make_request(r, req_id=None) -> Request:
    """Request from a structured record / dict with keys ox..gz, speed, depart, horizon."""
    def g(*names):
        for n in names:
            try:
                return r[n]
            except (KeyError, ValueError, IndexError):
                continue
        raise KeyError(names)
    rid = req_id if req_id is not None else int(g("req_id")) if _has(r, "req_id") else 0
    return Request(int(rid), float(g("ox")), float(g("oy")), float(g("oz")), float(g("gx")), float(g("gy")),
                   float(g("gz")), float(g("speed_mps", "speed")), int(g("depart_step", "depart")),
                   int(g("horizon")), 0)


# numpy mirrors of the ABI's request and result records (same offsets, natural alignment)
_REQ_NP = np.dtype({"names": [f for f, _ in Request._fields_],
                    "formats": ["<u8"] + ["<f8"] * 7 + ["<i8", "<i4", "<i4"],
                    "offsets": [getattr(Request, f).offset for f, _ in Request._fields_],
                    "itemsize": ctypes.sizeof(Request)})
_RES_FIELDS = [f for f, _ in Result._fields_ if f not in ("xyz", "actions")]
_RES_NP = np.dtype({"names": [f for f, _ in Result._fields_],
                    "formats": ["<i4", "<i4", "<u8", "<i4", "<i4", "<f8", "<f8", "<i4", "<i4", "<i4", "<i4",
                                "<u8", "<u8"],
                    "offsets": [getattr(Result, f).offset for f, _ in Result._fields_],
                    "itemsize": ctypes.sizeof(Result)})


def _requests(reqs):
    """ctypes array of n Requests. A structured numpy array with fields ox..gz, speed (or
    speed_mps), depart (or depart_step), horizon and optionally req_id is converted column
    by column; anything else record by record through make_request."""
    n = len(reqs)
    names = getattr(getattr(reqs, "dtype", None), "names", None) or ()
    speed = "speed_mps" if "speed_mps" in names else "speed"
    depart = "depart_step" if "depart_step" in names else "depart"
    if all(k in names for k in ("ox", "oy", "oz", "gx", "gy", "gz", speed, depart, "horizon")):
        arr = np.zeros(n, dtype=_REQ_NP)
        if "req_id" in names:
            arr["req_id"] = reqs["req_id"]
        for k in ("ox", "oy", "oz", "gx", "gy", "gz"):
            arr[k] = reqs[k]
        arr["speed_mps"] = reqs[speed]
        arr["depart_step"] = reqs[depart]
        arr["horizon"] = reqs["horizon"]
        return (Request * n).from_buffer(arr)
    return (Request * n)(*[make_request(reqs[i]) for i in range(n)])


def _results(res, n, xyz=None, acts=None):
    """Result dicts from a ctypes Result array; sample points as views of xyz / acts."""
    rv = np.frombuffer(res, dtype=_RES_NP, count=n)
    cols = [rv[k].tolist() for k in _RES_FIELDS]
    out = [dict(zip(_RES_FIELDS, vals)) for vals in zip(*cols)]
    if xyz is not None:
        npts = rv["n_points"].tolist()
        for i, d in enumerate(out):
            d["xyz"] = xyz[i, : npts[i]]
            d["actions"] = acts[i, : max(npts[i] - 1, 0)]
    return out


def _point_buffers(res, n, cap):
    """Per-request sample buffers [n][cap][3] and [n][cap], named in the results."""
    xyz = np.zeros((n, cap, 3), dtype=np.float32)
    acts = np.zeros((n, cap), dtype=np.uint8)
    rv = np.frombuffer(res, dtype=_RES_NP, count=n)
    rv["xyz"] = xyz.ctypes.data + np.arange(n, dtype=np.uint64) * np.uint64(cap * 12)
    rv["actions"] = acts.ctypes.data + np.arange(n, dtype=np.uint64) * np.uint64(cap)
    return xyz, acts


def _has(r, name):
    try:
        r[name]
        return True
    except (KeyError, ValueError, IndexError):
        return False


def _result_dict(res: Result, xyz=None, acts=None):
    d = {k: getattr(res, k) for k, _ in Result._fields_ if k not in ("xyz", "actions")}
    n = res.n_points
    if xyz is not None:
        d["xyz"] = xyz[:n].copy()
    if acts is not None:
        d["actions"] = acts[: max(n - 1, 0)].copy()
    return d


class Scheduler:
    """One FastMDP FCFS scheduler (one CUDA context's worth of device state)."""

    def __init__(self, box, dt, gamma, actions, sep, n_slices_window=4096, max_slots=4096, heightmap=None,
                 clearance=0.0, deck_value=1000.0, static_wells=None, combine=0, wells=None, goal_reward=200.0,
                 cluster_size=0, threads_per_cta=0, batch_size=0, full_scan=False, index_vmax_mps=0.0,
                 index_cell_m=0.0, index_stage_items=0, lookahead_W=1, batch_mode=0, pipe_rebuild_items=0):
        self._L = load()
        air = Airspace()
        air.x0, air.y0, air.z0, air.x1, air.y1, air.z1 = map(float, box)
        air.dt = float(dt)
        air.n_slices_window = int(n_slices_window)
        air.max_slots = int(max_slots)
        self._keep = []
        if heightmap is not None:
            hm = np.ascontiguousarray(heightmap, dtype=np.float32)
            self._keep.append(hm)
            air.heightmap = _ptr(hm, ctypes.c_float)
            air.hm_ny, air.hm_nx = hm.shape
        air.clearance_m = float(clearance)
        air.deck_value = float(deck_value)
        if static_wells is not None and len(static_wells):
            sw = np.ascontiguousarray(static_wells, dtype=np.float64).reshape(-1, 6)
            self._keep.append(sw)
            air.static_wells = _ptr(sw, ctypes.c_double)
            air.n_static_wells = sw.shape[0]
        acts = (Action * len(actions))(*[Action(float(a), float(c)) for a, c in actions])
        sp = Sep(float(sep[0]), float(sep[1]))
        opt = Options()
        self._L.fmdp_options_default(ctypes.byref(opt))
        opt.combine = int(combine)
        opt.goal_reward = float(goal_reward)
        opt.cluster_size = int(cluster_size)
        opt.threads_per_cta = int(threads_per_cta)
        opt.batch_size = int(batch_size)
        opt.full_scan = int(bool(full_scan))
        opt.index_vmax_mps = float(index_vmax_mps)
        opt.index_cell_m = float(index_cell_m)
        opt.index_stage_items = int(index_stage_items)
        opt.batch_mode = int(batch_mode)
        opt.pipe_rebuild_items = int(pipe_rebuild_items)
        opt.lookahead_W = int(lookahead_W)
        if wells is not None:
            warr = (Well * len(wells))(*[Well(*map(float, w)) for w in wells])
            self._keep.append(warr)
            opt.wells = ctypes.cast(warr, ctypes.POINTER(Well))
            opt.n_wells = len(wells)
        h = ctypes.c_void_p()
        st = self._L.fmdp_create(ctypes.byref(air), float(gamma), acts, len(actions), ctypes.byref(sp),
                                 ctypes.byref(opt), ctypes.byref(h))
        if st != 0:
            raise FmdpError(st, self._L.fmdp_last_error(None).decode())
        self._h = h
        self.n_actions = len(actions)

    @classmethod
    def from_scenario(cls, sc, add_plans=True, **kw):
        args = dict(box=sc.box, dt=sc.dt, gamma=sc.gamma, actions=sc.actions, sep=sc.sep,
                    n_slices_window=sc.n_slices_window, max_slots=sc.max_slots or 4096, heightmap=sc.heightmap,
                    clearance=sc.clearance, static_wells=sc.static_wells, goal_reward=sc.goal_reward)
        args.update(kw)
        s = cls(**args)
        if add_plans and sc.plans:
            s.add_plans([(p.t0, p.xyz) for p in sc.plans])
        return s

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._L.fmdp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st):
        if st != 0:
            raise FmdpError(st, self._L.fmdp_last_error(self._h).decode())

    def set_stream(self, stream_ptr):
        self._check(self._L.fmdp_set_stream(self._h, ctypes.c_void_p(stream_ptr or None)))

    # ------------------------------------------------------------ plans
    def add_plan(self, t0, xyz):
        xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
        pid = ctypes.c_uint64()
        self._check(self._L.fmdp_add_plan(self._h, int(t0), _ptr(xyz, ctypes.c_float), xyz.shape[0],
                                          ctypes.byref(pid)))
        return pid.value

    def add_plans(self, plans):
        if not plans:
            return np.zeros(0, dtype=np.uint64)
        t0 = np.array([int(t) for t, _ in plans], dtype=np.int64)
        pts = [np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 3) for _, x in plans]
        cnt = np.array([p.shape[0] for p in pts], dtype=np.int32)
        xyz = np.ascontiguousarray(np.concatenate(pts, axis=0))
        ids = np.zeros(len(plans), dtype=np.uint64)
        self._check(self._L.fmdp_add_plans(self._h, len(plans), _ptr(t0, ctypes.c_int64), _ptr(cnt, ctypes.c_int32),
                                           _ptr(xyz, ctypes.c_float), _ptr(ids, ctypes.c_uint64)))
        return ids

    def add_plans_packed(self, t0s, counts, xyz):
        """Known plans in the C ABI's packed form: plan i starts at step t0s[i] and holds
        counts[i] consecutive (x, y, z) samples of xyz (all plans back to back). The arrays
        are passed as they are when their dtypes already match (int64, int32, float32), so
        pinned host arrays are copied to the device directly."""
        t0s = np.ascontiguousarray(t0s, dtype=np.int64)
        counts = np.ascontiguousarray(counts, dtype=np.int32)
        xyz = np.ascontiguousarray(xyz, dtype=np.float32)
        if t0s.shape != counts.shape or t0s.ndim != 1 or xyz.size != 3 * int(counts.sum(dtype=np.int64)):
            raise ValueError("t0s and counts need one entry per plan, xyz 3 values per sample")
        ids = np.zeros(t0s.size, dtype=np.uint64)
        if t0s.size:
            self._check(self._L.fmdp_add_plans(self._h, t0s.size, _ptr(t0s, ctypes.c_int64),
                                               _ptr(counts, ctypes.c_int32), _ptr(xyz, ctypes.c_float),
                                               _ptr(ids, ctypes.c_uint64)))
        return ids

    def query_plans(self, t_begin, t_end):
        n = ctypes.c_int32()
        self._check(self._L.fmdp_query_plans(self._h, int(t_begin), int(t_end), None, 0, ctypes.byref(n)))
        ids = np.zeros(max(n.value, 1), dtype=np.uint64)
        self._check(self._L.fmdp_query_plans(self._h, int(t_begin), int(t_end), _ptr(ids, ctypes.c_uint64),
                                             ids.size, ctypes.byref(n)))
        return ids[: n.value]

    def save_plans(self, path):
        """Writes the plan table to a file (fmdp_save_plans); returns the plans written."""
        n = ctypes.c_int64()
        self._check(self._L.fmdp_save_plans(self._h, os.fsencode(path), ctypes.byref(n)))
        return n.value

    def load_plans(self, path, max_ids=1 << 22):
        """Adds the plans of a plan file as known plans (fmdp_load_plans); returns their new
        ids in file order (the first max_ids of them)."""
        ids = np.zeros(max_ids, dtype=np.uint64)
        n = ctypes.c_int64()
        self._check(self._L.fmdp_load_plans(self._h, os.fsencode(path), _ptr(ids, ctypes.c_uint64), max_ids,
                                            ctypes.byref(n)))
        return ids[:min(n.value, max_ids)].copy()

    def get_plan(self, pid):
        t0, n = ctypes.c_int64(), ctypes.c_int32()
        self._check(self._L.fmdp_get_plan(self._h, int(pid), ctypes.byref(t0), None, 0, ctypes.byref(n)))
        xyz = np.zeros((n.value, 3), dtype=np.float32)
        self._check(self._L.fmdp_get_plan(self._h, int(pid), ctypes.byref(t0), _ptr(xyz, ctypes.c_float), n.value,
                                          ctypes.byref(n)))
        return t0.value, xyz

    def expire(self, t_now):
        self._check(self._L.fmdp_expire(self._h, int(t_now)))

    def snapshot(self):
        self._check(self._L.fmdp_snapshot(self._h))

    def restore(self):
        self._check(self._L.fmdp_restore(self._h))

    def clear(self):
        self._check(self._L.fmdp_clear(self._h))

    # ------------------------------------------------------------ planning
    def schedule(self, req):
        r = make_request(req)
        cap = r.horizon + 1
        xyz = np.zeros((cap, 3), dtype=np.float32)
        acts = np.zeros(max(cap, 1), dtype=np.uint8)
        res = Result()
        res.xyz = _ptr(xyz, ctypes.c_float)
        res.actions = _ptr(acts, ctypes.c_uint8)
        self._check(self._L.fmdp_schedule(self._h, ctypes.byref(r), ctypes.byref(res)))
        return _result_dict(res, xyz, acts)

    def _many(self, fn, reqs, points=True):
        n = len(reqs)
        rq = _requests(reqs)
        res = (Result * n)()
        if not points:  # verdicts and counts only
            self._check(fn(self._h, rq, n, res))
            return _results(res, n)
        cap = int(np.frombuffer(rq, dtype=_REQ_NP, count=n)["horizon"].max(initial=0)) + 1
        xyz, acts = _point_buffers(res, n, cap)
        self._check(fn(self._h, rq, n, res))
        return _results(res, n, xyz, acts)

    def schedule_many(self, reqs, points=True):
        """FCFS in array order, one request after the other on the device."""
        return self._many(self._L.fmdp_schedule_many, reqs, points)

    def schedule_batch(self, reqs, points=True):
        """FCFS in array order through speculative batches; identical results."""
        return self._many(self._L.fmdp_schedule_batch, reqs, points)

    def serve(self, reqs, arrival_s, time_scale=1.0, max_in_flight=0, max_active_plans=0, expire_quantum=0,
              sim_start_step=None, points=True):
        """Continuous-batching serving run over an arrival trace (seconds after the call).
        Returns (results, latency_ms, report)."""
        n = len(reqs)
        rq = _requests(reqs)
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        assert arr.shape == (n,)
        o = ServeOptions()
        self._L.fmdp_serve_options_default(ctypes.byref(o))
        o.time_scale = float(time_scale)
        o.max_in_flight = int(max_in_flight)
        o.max_active_plans = int(max_active_plans)
        o.expire_quantum = int(expire_quantum)
        if sim_start_step is not None:
            o.sim_start_set = 1
            o.sim_start_step = int(sim_start_step)
        res = (Result * n)()
        cap = int(np.frombuffer(rq, dtype=_REQ_NP, count=n)["horizon"].max(initial=0)) + 1
        xyz, acts = _point_buffers(res, n, cap) if points else (None, None)
        lat = np.zeros(n, dtype=np.float64)
        rep = ServeReport()
        self._check(self._L.fmdp_serve(self._h, rq, _ptr(arr, ctypes.c_double), n, ctypes.byref(o), res,
                                       _ptr(lat, ctypes.c_double), ctypes.byref(rep)))
        out = _results(res, n, xyz, acts)
        return out, lat, {k: getattr(rep, k) for k, _ in ServeReport._fields_}

    # ---- learned proposal
    def learned_collect(self, reqs):
        """FastMDP rollouts of the requests against the table as it stands (nothing admitted);
        appends their (features, action) rows to the training set. Returns the row count."""
        n = len(reqs)
        rq = _requests(reqs)
        rows = ctypes.c_int32()
        self._check(self._L.fmdp_learned_collect(self._h, rq, n, ctypes.byref(rows)))
        return rows.value

    def learned_rows(self, max_rows):
        X = np.zeros((max_rows, 128), dtype=np.float32)
        y = np.zeros(max_rows, dtype=np.uint8)
        n = ctypes.c_int32()
        self._check(self._L.fmdp_learned_rows(self._h, _ptr(X, ctypes.c_float), _ptr(y, ctypes.c_uint8), max_rows,
                                              ctypes.byref(n)))
        return X[: n.value], y[: n.value]

    def learned_clear_rows(self):
        self._check(self._L.fmdp_learned_clear_rows(self._h))

    def learned_init(self, seed=1):
        self._check(self._L.fmdp_learned_init(self._h, int(seed)))

    def learned_set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self._L.fmdp_learned_set_params(self._h, _ptr(p, ctypes.c_float), p.size))

    def learned_get_params(self):
        p = np.zeros(MLP_PARAMS, dtype=np.float32)
        self._check(self._L.fmdp_learned_get_params(self._h, _ptr(p, ctypes.c_float), p.size))
        return p

    def learned_train(self, epochs=4, batch=256, lr=1e-3, seed=1):
        losses = np.zeros(max(epochs, 1), dtype=np.float32)
        self._check(self._L.fmdp_learned_train(self._h, int(epochs), int(batch), float(lr), int(seed),
                                               _ptr(losses, ctypes.c_float)))
        return losses[:epochs]

    def learned_loss_grad(self, X, y):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.uint8)
        loss = np.zeros(1, dtype=np.float32)
        g = np.zeros(MLP_PARAMS, dtype=np.float32)
        self._check(self._L.fmdp_learned_loss_grad(self._h, _ptr(X, ctypes.c_float), _ptr(y, ctypes.c_uint8),
                                                   X.shape[0], _ptr(loss, ctypes.c_float), _ptr(g, ctypes.c_float)))
        return float(loss[0]), g

    def learned_evaluate(self, reqs, slack=0.05):
        n = len(reqs)
        rq = _requests(reqs)
        rep = LearnedReport()
        acc = np.zeros(max(n, 1), dtype=np.int32)
        sp = np.zeros(max(n, 1), dtype=np.int32)
        sf = np.zeros(max(n, 1), dtype=np.int32)
        self._check(self._L.fmdp_learned_evaluate(self._h, rq, n, float(slack), ctypes.byref(rep),
                                                  _ptr(acc, ctypes.c_int32), _ptr(sp, ctypes.c_int32),
                                                  _ptr(sf, ctypes.c_int32)))
        return {k: getattr(rep, k) for k, _ in LearnedReport._fields_}, acc[:n], sp[:n], sf[:n]

    def selftest_wait_timeout(self):
        """Makes one bounded device wait run out on purpose; returns the status observed."""
        st = ctypes.c_int32(0)
        self._check(self._L.fmdp_selftest_wait_timeout(self._h, ctypes.byref(st)))
        return st.value

    def schedule_cosim(self, reqs, points=True):
        """The batch co-simulated on one clock (each request sees the others' wells), then
        admitted in array order."""
        return self._many(self._L.fmdp_schedule_cosim, reqs, points)

    def schedule_departures(self, reqs, delays, points=True, batched=False):
        """FCFS where each request takes the first admissible of its variants departing
        delays[d] steps later (planned together; with batched, the variants of many requests
        through speculative batches, same results). Returns (results, chosen, verdicts)."""
        n = len(reqs)
        dl = np.ascontiguousarray(delays, dtype=np.int64)
        D = dl.size
        chosen = np.zeros(max(n, 1), dtype=np.int32)
        verd = np.zeros((max(n, 1), max(D, 1)), dtype=np.int32)
        fn = self._L.fmdp_schedule_departures_batch if batched else self._L.fmdp_schedule_departures
        out = self._many(lambda h, rq, nn, res: fn(
            h, rq, nn, _ptr(dl, ctypes.c_int64), D, res, _ptr(chosen, ctypes.c_int32), _ptr(verd, ctypes.c_int32)),
            reqs, points)
        return out, chosen[:n], verd[:n, :D]

    def schedule_learned(self, reqs, slack=0.05, points=True):
        """FCFS where each request takes its accepted proposal, else its FastMDP plan."""
        n = len(reqs)
        rep = LearnedReport()
        out = self._many(lambda h, rq, nn, res: self._L.fmdp_schedule_learned(h, rq, nn, float(slack), res,
                                                                              ctypes.byref(rep)), reqs, points)
        return out, {k: getattr(rep, k) for k, _ in LearnedReport._fields_}

    def autotune(self, sample, force=False):
        """Times one wave of the sample's rollouts under each launch shape and caches the
        fastest for the current key; batched calls then use it."""
        n = len(sample)
        rq = _requests(sample) if n else (Request * 1)()
        rep = TuneReport()
        self._check(self._L.fmdp_autotune(self._h, rq, n, 1 if force else 0, ctypes.byref(rep)))
        out = {k: getattr(rep, k) for k, _ in TuneReport._fields_ if k != "chosen"}
        out["chosen"] = _entry_dict(rep.chosen)
        return out

    def tune_cache(self):
        n = ctypes.c_int32(0)
        self._check(self._L.fmdp_tune_cache_get(self._h, None, 0, ctypes.byref(n)))
        buf = (TuneEntry * max(n.value, 1))()
        self._check(self._L.fmdp_tune_cache_get(self._h, buf, n.value, ctypes.byref(n)))
        return [_entry_dict(buf[i]) for i in range(n.value)]

    def load_tune_cache(self, entries):
        n = len(entries)
        buf = (TuneEntry * max(n, 1))()
        for i, e in enumerate(entries):
            for k, _ in TuneEntry._fields_:
                setattr(buf[i], k, e[k])
        self._check(self._L.fmdp_tune_cache_put(self._h, buf, n))

    def stage(self, reqs):
        n = len(reqs)
        self._staged = _requests(reqs)
        self._check(self._L.fmdp_stage_requests(self._h, self._staged, n))

    def schedule_staged(self, batched=False):
        n = ctypes.c_int32()
        self._check(self._L.fmdp_schedule_staged(self._h, int(bool(batched)), ctypes.byref(n)))
        return n.value

    def fetch_staged(self):
        n = len(self._staged)
        cap = int(np.frombuffer(self._staged, dtype=_REQ_NP, count=n)["horizon"].max(initial=0)) + 1
        res = (Result * n)()
        xyz, acts = _point_buffers(res, n, cap)
        self._check(self._L.fmdp_fetch_staged(self._h, res, n))
        return _results(res, n, xyz, acts)

    def rollout_trace(self, req):
        r = make_request(req)
        cap = r.horizon + 1
        A = self.n_actions
        xyz = np.zeros((cap, 3), dtype=np.float32)
        acts = np.zeros(max(cap, 1), dtype=np.uint8)
        q = np.zeros((cap, A))
        states = np.zeros((cap, 3))
        heads = np.zeros(cap, dtype=np.int32)
        ties = np.zeros(max(cap, 1), dtype=np.uint8)
        res = Result()
        res.xyz = _ptr(xyz, ctypes.c_float)
        res.actions = _ptr(acts, ctypes.c_uint8)
        self._check(self._L.fmdp_rollout_trace(self._h, ctypes.byref(r), ctypes.byref(res), _ptr(q, ctypes.c_double),
                                               _ptr(states, ctypes.c_double), _ptr(heads, ctypes.c_int32),
                                               _ptr(ties, ctypes.c_uint8)))
        d = _result_dict(res, xyz, acts)
        n = res.n_points
        d.update(q=q[: n - 1], states=states[:n], headings=heads[:n],
                 ties=ties[: n - 1].astype(bool))
        return d

    def sep_check(self, t0, xyz):
        xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
        rep = SepReport()
        self._check(self._L.fmdp_sep_check(self._h, int(t0), _ptr(xyz, ctypes.c_float), xyz.shape[0],
                                           ctypes.byref(rep)))
        return {k: getattr(rep, k) for k, _ in SepReport._fields_}

    def sep_check_noalloc(self, t0, xyz):
        """fmdp_sep_check_noalloc: the same check using the library's fixed scratch array."""
        xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
        rep = SepReport()
        self._check(self._L.fmdp_sep_check_noalloc(self._h, int(t0), _ptr(xyz, ctypes.c_float), xyz.shape[0],
                                                   ctypes.byref(rep)))
        return {k: getattr(rep, k) for k, _ in SepReport._fields_}

    # ------------------------------------------------------------ profiling
    def set_profiling(self, on=True):
        self._check(self._L.fmdp_set_profiling(self._h, int(on)))

    def set_batch_mode(self, mode):
        """0: pipelined batches (default), 1: speculative waves; same results."""
        self._check(self._L.fmdp_set_batch_mode(self._h, int(mode)))

    def last_call_times(self):
        """Completion time of each request of the last scheduling call, ms from its start."""
        n = ctypes.c_int32()
        self._check(self._L.fmdp_last_call_times(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value)
        if n.value:
            self._check(self._L.fmdp_last_call_times(self._h, _ptr(out, ctypes.c_double), n.value, ctypes.byref(n)))
        return out

    def probe_peaks(self):
        """Measured FP32 FMA (TFLOP/s), MUFU rsqrt and exp2 (Top/s) rates and the SM clock."""
        pk = Peaks()
        self._check(self._L.fmdp_probe_peaks(self._h, ctypes.byref(pk)))
        return {k: getattr(pk, k) for k, _ in Peaks._fields_}

    def write_metrics(self, path, **tags):
        """Appends this context's statistics (fmdp_get_stats) and the given tags, with a
        wall-clock time stamp, as one JSON line to the file at path."""
        import time
        append_jsonl(path, {"time_unix_s": time.time(), "tags": tags, "stats": self.stats()})

    def stats(self):
        s = Stats()
        self._check(self._L.fmdp_get_stats(self._h, ctypes.byref(s)))
        d = {k: getattr(s, k) for k, _ in Stats._fields_ if k not in ("phase_cycles", "pipe_head_n", "pipe_head_s")}
        d["pipe_head_n"] = list(s.pipe_head_n)
        d["pipe_head_s"] = list(s.pipe_head_s)
        d["phase_cycles"] = list(s.phase_cycles)
        return d
