"""ctypes wrapper of the FP64 CPU FastMDP oracle.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The GPU scheduler never
imports this package, and this package never imports the scheduler.

The oracle is a plain, slow restatement of the paper's method in double precision
(see ``fmdp_oracle.c`` for the passage each step follows).
"""
import ctypes

import numpy as np

from .build_oracle import LIB_PATH, build

ORC_MAX_ACTIONS = 64
ORC_MAX_WELLS = 16

ADMITTED, REJ_CONFLICT, REJ_TERRAIN, REJ_HORIZON, REJ_NO_ACTION = range(5)

# Table 3 (peaks created in the environment), intruder row: magnitude -1000, decay .97,
# centre p + v t, radius 300 + 10 t, for t in {-5, 0, 5, 10, 15}.
PAPER_WELLS = tuple((float(t), 300.0 + 10.0 * t, 1000.0, 0.97) for t in (-5, 0, 5, 10, 15))


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
        ("x1", ctypes.c_double), ("y1", ctypes.c_double), ("z1", ctypes.c_double),
        ("dt", ctypes.c_double), ("gamma", ctypes.c_double), ("goal_reward", ctypes.c_double),
        ("deck_value", ctypes.c_double), ("clearance", ctypes.c_double),
        ("sep_h", ctypes.c_double), ("sep_v", ctypes.c_double),
        ("combine", ctypes.c_int32), ("n_actions", ctypes.c_int32),
        ("dpsi_deg", ctypes.c_double * ORC_MAX_ACTIONS), ("climb", ctypes.c_double * ORC_MAX_ACTIONS),
        ("n_wells", ctypes.c_int32),
        ("w_tau", ctypes.c_double * ORC_MAX_WELLS), ("w_radius", ctypes.c_double * ORC_MAX_WELLS),
        ("w_mag", ctypes.c_double * ORC_MAX_WELLS), ("w_gamma", ctypes.c_double * ORC_MAX_WELLS),
        ("hm_nx", ctypes.c_int32), ("hm_ny", ctypes.c_int32),
        ("heightmap", ctypes.POINTER(ctypes.c_float)),
        ("n_static", ctypes.c_int32),
        ("static_wells", ctypes.POINTER(ctypes.c_double)),
        ("lookahead_W", ctypes.c_int32),
    ]


class OrcRequest(ctypes.Structure):
    _fields_ = [("ox", ctypes.c_double), ("oy", ctypes.c_double), ("oz", ctypes.c_double),
                ("gx", ctypes.c_double), ("gy", ctypes.c_double), ("gz", ctypes.c_double),
                ("speed", ctypes.c_double), ("depart", ctypes.c_int64), ("horizon", ctypes.c_int32)]


class OrcResult(ctypes.Structure):
    _fields_ = [("verdict", ctypes.c_int32), ("n_points", ctypes.c_int32), ("captured", ctypes.c_int32),
                ("near_ties", ctypes.c_int32), ("followed_ties", ctypes.c_int32),
                ("mismatch_step", ctypes.c_int32), ("first_conflict", ctypes.c_int32),
                ("first_terrain", ctypes.c_int32), ("min_sep_h", ctypes.c_double),
                ("min_sep_v", ctypes.c_double), ("plan_id", ctypes.c_int64),
                ("well_tests", ctypes.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        dp, fp, ip = P(ctypes.c_double), P(ctypes.c_float), P(ctypes.c_int32)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [P(OrcParams)]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_add_plan.restype = ctypes.c_int64
        L.orc_add_plan.argtypes = [ctypes.c_void_p, ctypes.c_int64, fp, ctypes.c_int32]
        L.orc_n_plans.restype = ctypes.c_int32
        L.orc_n_plans.argtypes = [ctypes.c_void_p]
        L.orc_set_threads.argtypes = [ctypes.c_int32]
        L.orc_set_threads.restype = ctypes.c_int32
        L.orc_heading_table.argtypes = [ctypes.c_double] * 4 + [dp, dp]
        L.orc_terrain.restype = ctypes.c_double
        L.orc_terrain.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
        L.orc_q_values.restype = ctypes.c_int64
        L.orc_q_values.argtypes = [ctypes.c_void_p, dp, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                   dp, dp, dp, dp, dp, dp, dp, ip, dp]
        L.orc_rollout.restype = ctypes.c_int32
        L.orc_rollout.argtypes = [ctypes.c_void_p, P(OrcRequest), ip, ctypes.c_int32, ctypes.c_int32,
                                  fp, dp, ip, ip, dp, dp, ip, P(OrcResult)]
        L.orc_sep_check.restype = ctypes.c_int64
        L.orc_sep_check.argtypes = [ctypes.c_void_p, ctypes.c_int64, fp, ctypes.c_int32, P(OrcResult)]
        L.orc_cosim.restype = ctypes.c_int32
        L.orc_cosim.argtypes = [ctypes.c_void_p, P(OrcRequest), ctypes.c_int32, ip, ctypes.c_int32, fp, ip, dp, dp,
                                P(OrcResult)]
        L.orc_schedule.restype = ctypes.c_int32
        L.orc_schedule.argtypes = [ctypes.c_void_p, P(OrcRequest), ctypes.c_int32, fp, ip, P(OrcResult)]
        _lib = L
    return _lib


def set_threads(n):
    """Threads that value a rollout step's actions (OpenMP build); returns the number in
    effect. The results do not depend on it."""
    return int(lib().orc_set_threads(int(n)))


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


def _res_dict(r: OrcResult):
    return {k: getattr(r, k) for k, _ in OrcResult._fields_}


def heading_table(ox, oy, gx, gy):
    C = np.zeros(24)
    S = np.zeros(24)
    lib().orc_heading_table(ox, oy, gx, gy, _ptr(C, ctypes.c_double), _ptr(S, ctypes.c_double))
    return C, S


def make_request(req):
    """OrcRequest from a structured request record or a dict-like with the same keys."""
    return OrcRequest(float(req["ox"]), float(req["oy"]), float(req["oz"]), float(req["gx"]),
                      float(req["gy"]), float(req["gz"]), float(req["speed"]), int(req["depart"]),
                      int(req["horizon"]))


class Oracle:
    """FP64 CPU oracle of FastMDP FCFS planning over a database of known plans."""

    def __init__(self, box, dt, gamma, actions, sep, wells=PAPER_WELLS, combine=0, goal_reward=200.0,
                 heightmap=None, clearance=0.0, deck_value=1000.0, static_wells=None, lookahead_W=1):
        p = OrcParams()
        p.lookahead_W = int(lookahead_W)
        p.x0, p.y0, p.z0, p.x1, p.y1, p.z1 = map(float, box)
        p.dt, p.gamma, p.goal_reward = float(dt), float(gamma), float(goal_reward)
        p.deck_value, p.clearance = float(deck_value), float(clearance)
        p.sep_h, p.sep_v = map(float, sep)
        p.combine = int(combine)
        p.n_actions = len(actions)
        for i, (dpsi, climb) in enumerate(actions):
            p.dpsi_deg[i] = dpsi
            p.climb[i] = climb
        p.n_wells = len(wells)
        for i, (tau, rad, mag, gam) in enumerate(wells):
            p.w_tau[i], p.w_radius[i], p.w_mag[i], p.w_gamma[i] = tau, rad, mag, gam
        self._hm = None
        if heightmap is not None:
            self._hm = np.ascontiguousarray(heightmap, dtype=np.float32)
            p.hm_ny, p.hm_nx = self._hm.shape
            p.heightmap = _ptr(self._hm, ctypes.c_float)
        self._sw = None
        if static_wells is not None and len(static_wells):
            self._sw = np.ascontiguousarray(static_wells, dtype=np.float64).reshape(-1, 6)
            p.n_static = self._sw.shape[0]
            p.static_wells = _ptr(self._sw, ctypes.c_double)
        self.n_actions = len(actions)
        self.dt = float(dt)
        self._h = lib().orc_create(ctypes.byref(p))
        if not self._h:
            raise ValueError("oracle rejected its parameters")

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_destroy(self._h)
            self._h = None

    @classmethod
    def from_scenario(cls, sc, **kw):
        args = dict(box=sc.box, dt=sc.dt, gamma=sc.gamma, actions=sc.actions, sep=sc.sep,
                    goal_reward=sc.goal_reward, heightmap=sc.heightmap, clearance=sc.clearance,
                    static_wells=sc.static_wells)
        args.update(kw)
        o = cls(**args)
        for pl in sc.plans:
            o.add_plan(pl.t0, pl.xyz)
        return o

    def add_plan(self, t0, xyz):
        xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
        return int(lib().orc_add_plan(self._h, int(t0), _ptr(xyz, ctypes.c_float), xyz.shape[0]))

    @property
    def n_plans(self):
        return int(lib().orc_n_plans(self._h))

    def terrain(self, x, y):
        return float(lib().orc_terrain(self._h, float(x), float(y)))

    def q_values(self, s, h, t, speed, origin, goal):
        A = self.n_actions
        C, S = heading_table(origin[0], origin[1], goal[0], goal[1])
        s = np.asarray(s, dtype=np.float64)
        goal = np.asarray(goal, dtype=np.float64)
        out = {k: np.zeros(A) for k in ("Q", "g", "P", "V")}
        valid = np.zeros(A, dtype=np.int32)
        nxt = np.zeros(3 * A)
        tests = lib().orc_q_values(self._h, _ptr(s, ctypes.c_double), int(h), int(t), float(speed),
                                   _ptr(goal, ctypes.c_double), _ptr(C, ctypes.c_double), _ptr(S, ctypes.c_double),
                                   *(_ptr(out[k], ctypes.c_double) for k in ("Q", "g", "P", "V")),
                                   _ptr(valid, ctypes.c_int32), _ptr(nxt, ctypes.c_double))
        out.update(valid=valid.astype(bool), nxt=nxt.reshape(A, 3), tests=int(tests))
        return out

    def rollout(self, req, follow=None, trace=False):
        r = make_request(req)
        cap = r.horizon + 1
        A = self.n_actions
        xyz = np.zeros((cap, 3), dtype=np.float32)
        states = np.zeros((cap, 3))
        heads = np.zeros(cap, dtype=np.int32)
        acts = np.full(cap, -1, dtype=np.int32)
        qt = np.zeros((cap, A)) if trace else None
        st = np.zeros((cap, A)) if trace else None
        ties = np.zeros(cap, dtype=np.int32)
        fol = None
        nf = 0
        if follow is not None:
            fol = np.ascontiguousarray(follow, dtype=np.int32)
            nf = fol.size
        res = OrcResult()
        rc = lib().orc_rollout(self._h, ctypes.byref(r), _ptr(fol, ctypes.c_int32), nf, cap,
                               _ptr(xyz, ctypes.c_float), _ptr(states, ctypes.c_double),
                               _ptr(heads, ctypes.c_int32), _ptr(acts, ctypes.c_int32),
                               _ptr(qt, ctypes.c_double), _ptr(st, ctypes.c_double),
                               _ptr(ties, ctypes.c_int32), ctypes.byref(res))
        if rc != 0:
            raise ValueError("oracle rollout rejected the request")
        d = _res_dict(res)
        n = res.n_points
        d.update(xyz=xyz[:n], states=states[:n], headings=heads[:n], actions=acts[:n - 1],
                 ties=ties[:n - 1].astype(bool))
        if trace:
            d.update(q=qt[:n - 1], scale=st[:n - 1])
        return d

    def sep_check(self, t0, xyz):
        xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
        res = OrcResult()
        nconf = lib().orc_sep_check(self._h, int(t0), _ptr(xyz, ctypes.c_float), xyz.shape[0],
                                    ctypes.byref(res))
        d = _res_dict(res)
        d["conflicts"] = int(nconf)
        return {k: d[k] for k in ("first_conflict", "first_terrain", "min_sep_h", "min_sep_v", "conflicts")}

    def schedule(self, req):
        r = make_request(req)
        cap = r.horizon + 1
        xyz = np.zeros((cap, 3), dtype=np.float32)
        acts = np.full(cap, -1, dtype=np.int32)
        res = OrcResult()
        if lib().orc_schedule(self._h, ctypes.byref(r), cap, _ptr(xyz, ctypes.c_float),
                              _ptr(acts, ctypes.c_int32), ctypes.byref(res)) != 0:
            raise ValueError("oracle schedule rejected the request")
        d = _res_dict(res)
        n = res.n_points
        d.update(xyz=xyz[:n].copy(), actions=acts[:n - 1].copy())
        return d

    def schedule_departures(self, req, delays):
        """Departure-time candidates (Sec. I: a recommended take-off time among several
        candidates; Sec. IV: scheduling at different departure times). The variants of req
        departing delays[d] steps later are taken in the given order, each planned,
        checked and admitted or rejected exactly as by schedule(); the first admitted one
        ends the search (a rejected variant leaves the table as it was). Returns the index
        of the admitted variant (-1 when none) and the results of the variants tried."""
        fields = ("ox", "oy", "oz", "gx", "gy", "gz", "speed", "depart", "horizon")
        tried = []
        for d, delay in enumerate(delays):
            v = {k: req[k] for k in fields}
            v["depart"] = int(req["depart"]) + int(delay)
            res = self.schedule(v)
            tried.append(res)
            if res["verdict"] == ADMITTED:
                return d, tried
        return -1, tried

    def cosim(self, reqs, follow=None, trace=False):
        """Co-simulation of a batch on one clock (Alg. 1 with the batch's aircraft as
        each other's wells, Sec. V); nothing is admitted. follow: optional per-request
        action sequences taken at near-ties. Returns one dict per request."""
        n = len(reqs)
        rq = (OrcRequest * n)(*[make_request(r) for r in reqs])
        cap = max(int(r["horizon"]) for r in reqs) + 1
        A = self.n_actions
        xyz = np.zeros((n, cap, 3), dtype=np.float32)
        acts = np.full((n, cap), -1, dtype=np.int32)
        fol = None
        if follow is not None:
            fol = np.full((n, cap), -1, dtype=np.int32)
            for i, f in enumerate(follow):
                f = np.asarray(f, dtype=np.int32)
                fol[i, :f.size] = f
        qt = np.zeros((n, cap, A)) if trace else None
        st = np.zeros((n, cap, A)) if trace else None
        res = (OrcResult * n)()
        if lib().orc_cosim(self._h, rq, n, _ptr(fol, ctypes.c_int32), cap, _ptr(xyz, ctypes.c_float),
                           _ptr(acts, ctypes.c_int32), _ptr(qt, ctypes.c_double), _ptr(st, ctypes.c_double),
                           res) != 0:
            raise ValueError("oracle co-simulation rejected the requests")
        out = []
        for i in range(n):
            d = _res_dict(res[i])
            m = res[i].n_points
            d.update(xyz=xyz[i, :m].copy(), actions=acts[i, :m - 1].copy())
            if trace:
                d.update(q=qt[i, :m - 1].copy(), scale=st[i, :m - 1].copy())
            out.append(d)
        return out

    def schedule_cosim(self, reqs, follow=None):
        """Co-simulation, then first-come-first-served admission in array order: a
        captured trajectory is stored if it keeps separation from every stored plan
        (earlier members of the batch included) and clears the terrain."""
        out = self.cosim(reqs, follow)
        for r, d in zip(reqs, out):
            if d["captured"]:
                chk = self.sep_check(int(r["depart"]), d["xyz"])
                if chk["first_conflict"] >= 0:
                    d["verdict"] = REJ_CONFLICT
                elif chk["first_terrain"] >= 0:
                    d["verdict"] = REJ_TERRAIN
                else:
                    d["verdict"] = ADMITTED
                    self.add_plan(int(r["depart"]), d["xyz"])
                d.update(first_conflict=chk["first_conflict"], first_terrain=chk["first_terrain"],
                         min_sep_h=chk["min_sep_h"], min_sep_v=chk["min_sep_v"])
        return out
