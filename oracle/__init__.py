"""FP64 CPU oracle of the per-step vehicle update -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference arm may import
this package.  It wraps oracle/moss_oracle.c (plain C, FP64; single-threaded unless asked
for threads, whose count does not change any result) with ctypes
and shares no code with the CUDA library.  Readings R1-R14, R17 and R19 of the model are
listed at the top of moss_oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "moss_oracle.c")
_LIB = os.path.join(_HERE, "libmoss_oracle.so")

STATUS_WAIT, STATUS_ACTIVE, STATUS_DONE = 0, 1, 2


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "moss_oracle.h"))):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                               "-Wall", "-o", _LIB, _SRC, "-lm"])
    return _LIB


class _Net(C.Structure):
    _fields_ = [("n_lanes", C.c_int), ("n_edges", C.c_int), ("n_ctrl", C.c_int)] + [
        (f, C.c_void_p) for f in (
            "lane_len", "lane_edge", "lane_index", "lane_left", "lane_right",
            "succ_off", "succ_lane", "succ_edge", "lane_ctrl", "lane_group",
            "ctrl_offset", "ctrl_green", "ctrl_yellow", "ctrl_nphase",
            "edge_nlanes", "edge_lane0")]


class _Params(C.Structure):
    _fields_ = [(f, C.c_double) for f in (
        "dt", "veh_len", "a", "b", "T", "s0", "p", "th", "bsafe", "p_lc", "a_min", "v_max",
        "d_look", "x_lc_min", "x_lc_end")] + [("window", C.c_int), ("n_windows", C.c_int),
                                             ("seed", C.c_uint64), ("th_jitter", C.c_double),
                                             ("signal_mode", C.c_int), ("mp_interval", C.c_int)]


_DBG_INT = ("active_before", "lead_kind", "lead_id")
_DBG_FIELDS = [("active_before", "i"), ("lead_kind", "i"), ("lead_id", "i"), ("s_own", "d"),
               ("vl_own", "d"), ("a_own", "d"), ("lc_dir", "i"), ("lc_cand", "i"),
               ("tau_lead", "i"), ("tau_foll", "i"), ("old_foll", "i"), ("incentive", "d"),
               ("a_use", "d"), ("flag", "i"), ("inserted", "i"),
               # R19 learned lane change: per trip, logits 3 per trip, inputs 16 per trip
               ("lc_learn", "i"), ("lc_margin", "d"), ("lc_logit", "d3"), ("lc_feat", "d16"),
               ("lc_near", "i")]


class _Debug(C.Structure):
    _fields_ = [(f, C.c_void_p) for f, _ in _DBG_FIELDS]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.or_create.restype = C.c_void_p
        lib.or_create.argtypes = [C.POINTER(_Net), C.POINTER(_Params), C.c_int] + [C.c_void_p] * 7
        lib.or_destroy.argtypes = [C.c_void_p]
        lib.or_step.argtypes = [C.c_void_p, C.c_void_p]
        lib.or_step.restype = C.c_int
        lib.or_run.argtypes = [C.c_void_p, C.c_int]
        lib.or_run.restype = C.c_int
        lib.or_get_state.argtypes = [C.c_void_p] + [C.c_void_p] * 7
        lib.or_set_state.argtypes = [C.c_void_p] + [C.c_void_p] * 6 + [C.c_int]
        lib.or_get_metrics.argtypes = [C.c_void_p] * 4
        lib.or_signal_state.argtypes = [C.c_void_p, C.c_int, C.c_int]
        lib.or_signal_state.restype = C.c_int
        lib.or_splitmix64.argtypes = [C.c_uint64]
        lib.or_splitmix64.restype = C.c_uint64
        lib.or_neighbors.argtypes = [C.c_void_p, C.c_void_p]
        lib.or_departure_lane.argtypes = [C.c_void_p, C.c_int]
        lib.or_departure_lane.restype = C.c_int
        lib.or_get_ctrl_state.argtypes = [C.c_void_p, C.c_void_p]
        lib.or_set_ctrl_state.argtypes = [C.c_void_p, C.c_void_p]
        lib.or_set_lane_limits.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.or_set_links.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
        lib.or_set_links.restype = C.c_int
        lib.or_set_threads.argtypes = [C.c_void_p, C.c_int]
        lib.or_set_threads.restype = None
        lib.or_set_lc_model.argtypes = [C.c_void_p, C.c_void_p, C.c_double]
        lib.or_set_lc_model.restype = C.c_int
        lib.or_bf16.argtypes = [C.c_double]
        lib.or_bf16.restype = C.c_double
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def splitmix64(z: int) -> int:
    return int(_load().or_splitmix64(C.c_uint64(z & 0xFFFFFFFFFFFFFFFF)))


def bf16(x: float) -> float:
    """The oracle's BF16 rounding (nearest, ties to even) of one value."""
    return float(_load().or_bf16(float(x)))


class Oracle:
    """One simulation instance.  `net` and `dem` are synth.Network / synth.Demand (or any
    objects with the same array attributes); `params` a dict like synth.default_params()."""

    def __init__(self, net, dem, params: dict, n_windows: int = 1, threads: int = 1):
        lib = _load()
        i32 = lambda a: np.ascontiguousarray(a, np.int32)
        self._keep = []

        def k(a):
            self._keep.append(a)
            return _p(a)
        self.n_lanes = net.n_lanes
        self.n_ctrl = net.n_ctrl
        self.n = dem.n
        self.n_windows = n_windows
        self.net_c = _Net(net.n_lanes, net.n_edges, net.n_ctrl,
                          k(np.ascontiguousarray(net.lane_len, np.float32)),
                          *[k(i32(getattr(net, f))) for f in (
                              "lane_edge", "lane_index", "lane_left", "lane_right",
                              "succ_off", "succ_lane", "succ_edge", "lane_ctrl", "lane_group",
                              "ctrl_offset", "ctrl_green", "ctrl_yellow", "ctrl_nphase",
                              "edge_nlanes", "edge_lane0")])
        p = params
        self.params = dict(p)
        self.par_c = _Params(p["dt"], p["veh_len"], p["idm_a"], p["idm_b"], p["idm_T"], p["idm_s0"],
                             p["mobil_p"], p["mobil_th"], p["mobil_bsafe"], p["p_lc"], p["a_min"],
                             p["v_max"], p["d_look"], p["x_lc_min"], p["x_lc_end"],
                             int(p["window"]), int(n_windows), int(p["seed"]),
                             float(p.get("mobil_th_jitter", 0.0)),
                             int(p.get("signal_mode", 0)), int(p.get("mp_interval", 10)))
        self.t_dep = i32(dem.t_dep)
        self.v0 = np.ascontiguousarray(dem.v0, np.float32)
        self.route_off = np.ascontiguousarray(dem.route_off, np.int64)
        self.route_edges = i32(dem.route_edges)
        lane = i32(dem.lane)
        x = np.ascontiguousarray(dem.x, np.float32)
        v = np.ascontiguousarray(dem.v, np.float32)
        self._keep += [self.t_dep, self.v0, self.route_off, self.route_edges, lane, x, v]
        self.h = lib.or_create(C.byref(self.net_c), C.byref(self.par_c), dem.n, _p(self.t_dep),
                               _p(self.v0), _p(self.route_off), _p(self.route_edges),
                               _p(lane), _p(x), _p(v))
        self.threads = max(1, int(threads))
        lib.or_set_threads(self.h, self.threads)

    def __del__(self):
        if getattr(self, "h", None):
            _load().or_destroy(self.h)
            self.h = None

    def step(self, debug: bool = False):
        lib = _load()
        if not debug:
            return lib.or_step(self.h, None), None
        arrs = {f: np.zeros(self.n * (int(t[1:]) if len(t) > 1 else 1), np.int32 if t == "i" else np.float64)
                for f, t in _DBG_FIELDS}
        dbg = _Debug(*[_p(arrs[f]) for f, _ in _DBG_FIELDS])
        err = lib.or_step(self.h, C.byref(dbg))
        arrs["lc_logit"] = arrs["lc_logit"].reshape(self.n, 3)
        arrs["lc_feat"] = arrs["lc_feat"].reshape(self.n, 16)
        return err, arrs

    def run(self, n_steps: int) -> int:
        return _load().or_run(self.h, n_steps)

    def state(self) -> dict:
        n = self.n
        st = dict(status=np.zeros(n, np.int32), lane=np.zeros(n, np.int32), x=np.zeros(n),
                  v=np.zeros(n), rp=np.zeros(n, np.int32), t_arr=np.zeros(n, np.int32))
        t = C.c_int(0)
        _load().or_get_state(self.h, _p(st["status"]), _p(st["lane"]), _p(st["x"]), _p(st["v"]),
                             _p(st["rp"]), _p(st["t_arr"]), C.byref(t))
        st["t"] = t.value
        return st

    def set_state(self, status, lane, x, v, rp, t, t_arr=None):
        a = [np.ascontiguousarray(status, np.int32), np.ascontiguousarray(lane, np.int32),
             np.ascontiguousarray(x, np.float64), np.ascontiguousarray(v, np.float64),
             np.ascontiguousarray(rp, np.int32)]
        ta = None if t_arr is None else np.ascontiguousarray(t_arr, np.int32)
        _load().or_set_state(self.h, *[_p(b) for b in a], None if ta is None else _p(ta), int(t))

    def metrics(self):
        m = self.n_windows * self.n_lanes
        vs = np.zeros(m)
        vc = np.zeros(m, np.int64)
        ctr = np.zeros(4, np.int64)
        _load().or_get_metrics(self.h, _p(vs), _p(vc), _p(ctr))
        return dict(vsum=vs.reshape(self.n_windows, self.n_lanes),
                    vcnt=vc.reshape(self.n_windows, self.n_lanes),
                    inserted=int(ctr[0]), arrived=int(ctr[1]), sum_tt=int(ctr[2]), errors=int(ctr[3]))

    def signal_state(self, lane: int, t: int) -> int:
        return _load().or_signal_state(self.h, lane, t)

    def ctrl_state(self) -> np.ndarray:
        """Max-pressure controller state (R13): [n_ctrl, 3] = green phase, pending phase
        (-1 none), step at which the pending phase turns green."""
        out = np.zeros((max(1, self.n_ctrl), 3), np.int32)
        _load().or_get_ctrl_state(self.h, _p(out))
        return out[:self.n_ctrl]

    def set_lane_limits(self, lanes, vmax=None, closed=None) -> None:
        """R14: speed limits (<= 0 / inf: none) and closures for the given lanes."""
        ln = np.ascontiguousarray(lanes, np.int32)
        vm = None if vmax is None else np.ascontiguousarray(vmax, np.float32)
        cl = None if closed is None else np.ascontiguousarray(closed, np.int32)
        _load().or_set_lane_limits(self.h, int(ln.shape[0]), _p(ln), None if vm is None else _p(vm),
                                   None if cl is None else _p(cl))

    def set_lane_links(self, lanes, open_mask) -> None:
        """R17: bit j of open_mask[k] opens (1) or closes (0) the j-th lane link of edge lane
        lanes[k].  The caller keeps every remaining route lane-connected."""
        ln = np.ascontiguousarray(lanes, np.int32)
        mk = np.ascontiguousarray(open_mask, np.uint32)
        assert ln.shape == mk.shape
        if _load().or_set_links(self.h, int(ln.shape[0]), _p(ln), _p(mk)) != 0:
            raise ValueError("or_set_links: internal or out-of-range lane, or more than 32 links")

    def set_lc_model(self, theta=None, margin: float = 0.2) -> None:
        """R19: decide discretionary lane changes with the learned network (theta: 5443
        floats in the C ABI's layout); None returns to the rule alone."""
        if theta is None:
            self._theta = None
            _load().or_set_lc_model(self.h, None, 0.0)
            return
        self._theta = np.ascontiguousarray(theta, np.float32)
        assert self._theta.shape == (5443,)
        if _load().or_set_lc_model(self.h, _p(self._theta), float(margin)) != 0:
            raise ValueError("margin outside [0, 1]")

    def set_ctrl_state(self, cs) -> None:
        cs = np.ascontiguousarray(np.asarray(cs, np.int32).reshape(-1, 3))
        assert cs.shape[0] == self.n_ctrl
        _load().or_set_ctrl_state(self.h, _p(cs))

    def neighbors(self) -> np.ndarray:
        out = np.zeros(6 * self.n, np.int32)
        _load().or_neighbors(self.h, _p(out))
        return out.reshape(self.n, 6)

    def departure_lane(self, trip: int) -> int:
        return _load().or_departure_lane(self.h, trip)
