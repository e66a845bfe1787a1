"""Python binding of the C ABI in include/moss103.h (argument marshalling only).

Every step of the simulation runs in libmoss103.so's CUDA kernels; this module only packs
numpy arrays / torch tensors into the C structs.  If the library is missing, importing
`load()` raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmoss103.so")

MS_OK, MS_ERR_ARG, MS_ERR_ROUTE, MS_ERR_CAPACITY, MS_ERR_CUDA, MS_ERR_DEVICE, MS_ERR_STATE = 0, -1, -2, -3, -4, -5, -6
ERR_NAMES = {0: "OK", -1: "ARG", -2: "ROUTE", -3: "CAPACITY", -4: "CUDA", -5: "DEVICE", -6: "STATE"}
SYMBOLS = ("ms_create", "ms_load_network", "ms_add_vehicles", "ms_step", "ms_step_timed", "ms_step_noalloc",
           "ms_load_network_batch", "ms_add_vehicles_batch", "ms_batch_offsets", "ms_autotune",
           "ms_set_lc_log", "ms_set_lc_model", "ms_set_lane_limits", "ms_set_lane_links", "ms_route_trips",
           "ms_sample_trips", "ms_sample_trips_radiation",
           "ms_read_lc_stats",
           "ms_mlp_train_step", "ms_mlp_train_step_tc",
           "ms_mlp_grad", "ms_mlp_grad_tc", "ms_test_tc_timeout", "ms_test_withhold_copies",
           "ms_mlp_predict",
           "ms_sync", "ms_read_state", "ms_read_state_async", "ms_read_wait",
           "ms_write_state", "ms_read_metrics", "ms_read_debug", "ms_last_error", "ms_destroy")


class ms_params(C.Structure):
    _fields_ = [(f, C.c_float) for f in (
        "dt", "veh_len", "idm_a", "idm_b", "idm_T", "idm_s0", "mobil_p", "mobil_th", "mobil_bsafe",
        "p_lc", "a_min", "v_max", "d_look", "x_lc_min", "x_lc_end")] + [
        ("window", C.c_int), ("n_windows", C.c_int), ("seed", C.c_uint64), ("debug", C.c_int),
        ("block", C.c_int), ("id_base", C.c_int), ("mobil_th_jitter", C.c_float),
        ("signal_mode", C.c_int), ("mp_interval", C.c_int)]


class ms_network(C.Structure):
    _fields_ = [("n_lanes", C.c_int), ("n_edges", C.c_int), ("n_ctrl", C.c_int)] + [
        (f, C.c_void_p) for f in (
            "lane_len", "lane_edge", "lane_index", "lane_left", "lane_right", "succ_off",
            "succ_lane", "succ_edge", "lane_ctrl", "lane_group", "ctrl_offset", "ctrl_green",
            "ctrl_yellow", "ctrl_nphase", "edge_nlanes", "edge_lane0")]


class ms_vehicles(C.Structure):
    _fields_ = [("n", C.c_int)] + [(f, C.c_void_p) for f in (
        "t_dep", "v0", "route_off", "route_edges", "lane", "x", "v")]


class ms_state(C.Structure):
    _fields_ = [("capacity", C.c_int), ("n_active", C.c_int), ("t", C.c_int)] + [
        (f, C.c_void_p) for f in ("id", "lane", "route_idx", "x", "v", "trip_status", "t_arr", "ctrl_state")]


class ms_metrics(C.Structure):
    _fields_ = [("lane_vsum", C.c_void_p), ("lane_vcnt", C.c_void_p), ("inserted", C.c_int64),
                ("arrived", C.c_int64), ("sum_travel_time", C.c_int64), ("n_active", C.c_int),
                ("t", C.c_int), ("movers_last_step", C.c_int), ("err", C.c_uint)]


_DBG_I = ("active_before", "lead_kind", "lead_id", "lc_dir", "lc_cand", "tau_lead", "tau_foll",
          "old_foll", "flag", "inserted")
_DBG_F = ("s_own", "vl_own", "a_own", "incentive", "a_use")
_DBG_LC = ("lc_learn", "lc_margin", "lc_logit", "lc_feat")   # learned lane change


class ms_debug(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in _DBG_I + _DBG_F + _DBG_LC]


_lib = None


def load():
    """Load libmoss103.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} not built: run paper_2405_12520_b300.build.build()")
        lib = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        lib.ms_create.argtypes = [C.POINTER(vp), C.POINTER(ms_params), vp]
        lib.ms_load_network.argtypes = [vp, C.POINTER(ms_network)]
        lib.ms_add_vehicles.argtypes = [vp, C.POINTER(ms_vehicles)]
        lib.ms_step.argtypes = [vp, C.c_int]
        lib.ms_step_timed.argtypes = [vp, C.c_int, C.POINTER(C.c_float)]
        lib.ms_step_noalloc.argtypes = [vp, C.c_int]
        lib.ms_load_network_batch.argtypes = [vp, C.c_int, C.POINTER(ms_network)]
        lib.ms_add_vehicles_batch.argtypes = [vp, C.c_int, C.POINTER(ms_vehicles)]
        lib.ms_batch_offsets.argtypes = [vp, vp, vp]
        lib.ms_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_float), vp]
        lib.ms_set_lc_log.argtypes = [vp, vp, vp, C.c_int, vp]
        lib.ms_set_lc_model.argtypes = [vp, vp, C.c_float]
        lib.ms_set_lane_limits.argtypes = [vp, C.c_int, vp, vp, vp]
        lib.ms_set_lane_links.argtypes = [vp, C.c_int, vp, vp]
        lib.ms_route_trips.argtypes = [vp, C.c_int, vp, vp, vp, vp, C.c_int64, vp]
        lib.ms_sample_trips.argtypes = [vp, C.c_int, vp, vp, C.c_int, C.c_int, C.c_int, C.c_uint64, vp, vp, vp]
        lib.ms_sample_trips_radiation.argtypes = [vp, C.c_int, vp, vp, C.c_int, C.c_int, C.c_uint64, vp, vp, vp]
        lib.ms_read_lc_stats.argtypes = [vp, vp]
        lib.ms_mlp_train_step.argtypes = [vp, vp, vp, C.c_int, vp, vp, vp, C.c_int, C.c_float, vp, vp, vp, vp]
        lib.ms_mlp_train_step_tc.argtypes = lib.ms_mlp_train_step.argtypes
        lib.ms_mlp_grad.argtypes = [vp, vp, vp, C.c_int, vp, vp, vp, vp, vp]
        lib.ms_mlp_grad_tc.argtypes = lib.ms_mlp_grad.argtypes
        lib.ms_test_tc_timeout.argtypes = [vp, vp, vp, C.c_int, vp, vp, vp, vp]
        lib.ms_test_withhold_copies.argtypes = [vp, C.c_int]
        lib.ms_mlp_predict.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, vp]
        lib.ms_sync.argtypes = [vp]
        lib.ms_read_state.argtypes = [vp, C.POINTER(ms_state), C.c_int]
        lib.ms_read_state_async.argtypes = [vp, C.POINTER(ms_state)]
        lib.ms_read_wait.argtypes = [vp, vp, vp]
        lib.ms_write_state.argtypes = [vp, C.POINTER(ms_state)]
        lib.ms_read_metrics.argtypes = [vp, C.POINTER(ms_metrics)]
        lib.ms_read_debug.argtypes = [vp, C.POINTER(ms_debug)]
        lib.ms_last_error.argtypes = [vp]
        lib.ms_last_error.restype = C.c_char_p
        lib.ms_destroy.argtypes = [vp]
        lib.ms_destroy.restype = None
        for f in SYMBOLS:
            if f not in ("ms_last_error", "ms_destroy"):
                getattr(lib, f).restype = C.c_int
        _lib = lib
    return _lib


MLP_NPARAM = 5443
MLP_WORK_FLOATS = 12096
LC_STAT_NAMES = ("candidates", "fallbacks", "agree") + tuple(f"conf_{r}{f}" for r in "slr" for f in "slr")


def _dp(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _st(stream):
    if stream is None:
        return None
    return C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)


def mlp_train_step(x, y, idx, theta, m, v, t, lr, class_w, work, stream=None, want_loss=False, tc=False):
    """One Adam step of the surrogate on device tensors (x bf16 [n,16], y int32, idx int32,
    theta/m/v float32 [5443], work float32 [MLP_WORK_FLOATS]); returns the loss if asked.
    tc: on the tcgen05 tensor cores (ms_mlp_train_step_tc) instead of mma.sync."""
    lib = load()
    name = "ms_mlp_train_step_tc" if tc else "ms_mlp_train_step"
    cw = np.ascontiguousarray(class_w, np.float32)
    loss = C.c_float(0.0)
    rc = getattr(lib, name)(_dp(x), _dp(y), _dp(idx), int(idx.numel()), _dp(theta), _dp(m), _dp(v), int(t),
                            float(lr), _p(cw), _dp(work), C.byref(loss) if want_loss else None, _st(stream))
    if rc:
        raise MossError(rc, name)
    return loss.value if want_loss else None


def test_tc_timeout(x, y, idx, theta, class_w, work, stream=None):
    """The tcgen05 gradient with no MMA issued (its first wait runs out): the return code,
    MS_ERR_DEVICE when the kernel reported the timeout."""
    lib = load()
    cw = np.ascontiguousarray(class_w, np.float32)
    return lib.ms_test_tc_timeout(_dp(x), _dp(y), _dp(idx), int(idx.numel()), _dp(theta), _p(cw), _dp(work),
                                  _st(stream))


def mlp_grad(x, y, idx, theta, class_w, work, grad, stream=None, tc=False):
    lib = load()
    name = "ms_mlp_grad_tc" if tc else "ms_mlp_grad"
    cw = np.ascontiguousarray(class_w, np.float32)
    rc = getattr(lib, name)(_dp(x), _dp(y), _dp(idx), int(idx.numel()), _dp(theta), _p(cw), _dp(work), _dp(grad),
                            _st(stream))
    if rc:
        raise MossError(rc, name)


def mlp_predict(x, theta, work, cls, margin, stream=None, logits=None):
    lib = load()
    rc = lib.ms_mlp_predict(_dp(x), int(x.shape[0]), _dp(theta), _dp(work), _dp(cls), _dp(margin), _dp(logits),
                            _st(stream))
    if rc:
        raise MossError(rc, "ms_mlp_predict")


class MossError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def params_struct(params: dict, debug: bool = False, n_windows: int = 1, block: int = 0,
                  id_base: int = 0) -> ms_params:
    p = params
    return ms_params(p["dt"], p["veh_len"], p["idm_a"], p["idm_b"], p["idm_T"], p["idm_s0"],
                     p["mobil_p"], p["mobil_th"], p["mobil_bsafe"], p["p_lc"], p["a_min"], p["v_max"],
                     p["d_look"], p["x_lc_min"], p["x_lc_end"], int(p["window"]), int(n_windows),
                     int(p["seed"]) & 0xFFFFFFFFFFFFFFFF, int(debug), int(block), int(id_base),
                     float(p.get("mobil_th_jitter", 0.0)), int(p.get("signal_mode", 0)),
                     int(p.get("mp_interval", 10)))


def _export_capacity(*tensors) -> int:
    """Elements every given export buffer can hold: the smallest length among them (the
    library writes up to that many 4-byte values into each)."""
    given = [t for t in tensors if t is not None]
    if not given:
        raise ValueError("no export buffer given")
    for t in given:
        if t.element_size() != 4 or not t.is_contiguous():
            raise ValueError("export buffers must be contiguous 4-byte tensors (float32 / int32)")
    return min(int(t.numel()) for t in given)


class Sim:
    """One simulation on the current CUDA device.

    Mirrors the C ABI: create (constructor), load_network, add_vehicles, step, sync,
    read_state, write_state, read_metrics, read_debug, last_error, destroy."""

    def __init__(self, params: dict, stream=None, debug: bool = False, n_windows: int = 1, block: int = 0,
                 id_base: int = 0):
        self.lib = load()
        self.h = C.c_void_p()
        self.params = dict(params)
        self.n_windows = n_windows
        self._p = params_struct(params, debug, n_windows, block, id_base)
        st = None
        if stream is not None:
            st = C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        self._check(self.lib.ms_create(C.byref(self.h), C.byref(self._p), st), "ms_create")
        self.n_lanes = 0
        self.n_trips = 0

    def _check(self, rc, what):
        if rc != MS_OK:
            msg = self.lib.ms_last_error(self.h).decode() if self.h else what
            raise MossError(rc, f"{what}: {msg}")

    def last_error(self) -> str:
        return self.lib.ms_last_error(self.h).decode()

    @staticmethod
    def _net_struct(net, keep):
        i32 = lambda a: np.ascontiguousarray(a, np.int32)
        arrs = [np.ascontiguousarray(net.lane_len, np.float32)] + [i32(getattr(net, f)) for f in (
            "lane_edge", "lane_index", "lane_left", "lane_right", "succ_off", "succ_lane", "succ_edge",
            "lane_ctrl", "lane_group", "ctrl_offset", "ctrl_green", "ctrl_yellow", "ctrl_nphase",
            "edge_nlanes", "edge_lane0")]
        keep += arrs
        return ms_network(int(net.n_lanes), int(net.n_edges), int(net.n_ctrl), *[_p(a) for a in arrs])

    @staticmethod
    def _veh_struct(dem, keep):
        arrs = [np.ascontiguousarray(dem.t_dep, np.int32), np.ascontiguousarray(dem.v0, np.float32),
                np.ascontiguousarray(dem.route_off, np.int64), np.ascontiguousarray(dem.route_edges, np.int32),
                np.ascontiguousarray(dem.lane, np.int32), np.ascontiguousarray(dem.x, np.float32),
                np.ascontiguousarray(dem.v, np.float32)]
        keep += arrs
        return ms_vehicles(int(dem.n), *[_p(a) for a in arrs])

    def load_network(self, net):
        keep = []
        s = self._net_struct(net, keep)
        self._check(self.lib.ms_load_network(self.h, C.byref(s)), "ms_load_network")
        self.n_lanes = int(net.n_lanes)
        self.n_ctrl = int(net.n_ctrl)

    def add_vehicles(self, dem):
        keep = []
        s = self._veh_struct(dem, keep)
        self._check(self.lib.ms_add_vehicles(self.h, C.byref(s)), "ms_add_vehicles")
        self.n_trips = int(dem.n)

    def load_network_batch(self, nets):
        keep = []
        arr = (ms_network * len(nets))(*[self._net_struct(n, keep) for n in nets])
        self._check(self.lib.ms_load_network_batch(self.h, len(nets), arr), "ms_load_network_batch")
        self.n_lanes = int(sum(n.n_lanes for n in nets))
        self.n_ctrl = int(sum(n.n_ctrl for n in nets))
        self.n_scen = len(nets)

    def add_vehicles_batch(self, dems):
        keep = []
        arr = (ms_vehicles * len(dems))(*[self._veh_struct(d, keep) for d in dems])
        self._check(self.lib.ms_add_vehicles_batch(self.h, len(dems), arr), "ms_add_vehicles_batch")
        self.n_trips = int(sum(d.n for d in dems))

    def batch_offsets(self):
        lo = np.zeros(self.n_scen + 1, np.int32)
        to = np.zeros(self.n_scen + 1, np.int32)
        self._check(self.lib.ms_batch_offsets(self.h, _p(lo), _p(to)), "ms_batch_offsets")
        return lo, to

    def autotune(self, trial_steps: int = 5):
        """Pick the fastest launch shape; returns (best ms per step, (block, decide grid
        factor, apply grid factor, lane-scan threads per tile, bucket block, bucket grid
        factor))."""
        ms = C.c_float()
        cfg = np.zeros(6, np.int32)
        self._check(self.lib.ms_autotune(self.h, int(trial_steps), C.byref(ms), _p(cfg)), "ms_autotune")
        return ms.value, tuple(int(c) for c in cfg)

    def step(self, n: int = 1):
        self._check(self.lib.ms_step(self.h, int(n)), "ms_step")

    def step_noalloc(self, n: int = 1):
        """ms_step_noalloc: the same steps as step(), allocating no device memory (lane-scan
        status in the library's static device array; calls must not overlap on the GPU)."""
        self._check(self.lib.ms_step_noalloc(self.h, int(n)), "ms_step_noalloc")

    def step_timed(self, n: int = 1) -> np.ndarray:
        """Run n steps kernel by kernel; device milliseconds per kernel
        (decide, lanes, bucket, apply) summed over the n steps."""
        ms = (C.c_float * 4)()
        self._check(self.lib.ms_step_timed(self.h, int(n), ms), "ms_step_timed")
        return np.array(list(ms), np.float64)

    def read_state_host(self, x, v, lane, vid) -> int:
        """Copy the vehicle state into caller-owned (e.g. pinned) host buffers given as
        torch CPU tensors; returns the number of active vehicles."""
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        cap = _export_capacity(x, v, lane, vid)
        s = ms_state(cap, 0, 0, ptr(vid), ptr(lane), None, ptr(x), ptr(v), None, None)
        self._check(self.lib.ms_read_state(self.h, C.byref(s), 0), "ms_read_state")
        return s.n_active

    def read_state_async(self, x, v, lane, vid):
        """Start an export of the vehicle state into pinned torch CPU tensors (any may be
        None) without synchronising; finish it with read_wait.  The tensors must stay alive
        and untouched until then."""
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        cap = _export_capacity(x, v, lane, vid)
        s = ms_state(cap, 0, 0, ptr(vid), ptr(lane), None, ptr(x), ptr(v), None, None)
        self._check(self.lib.ms_read_state_async(self.h, C.byref(s)), "ms_read_state_async")

    def read_wait(self) -> tuple:
        """Wait for the export started by read_state_async; returns (n_active, t)."""
        n, t = C.c_int(0), C.c_int(0)
        self._check(self.lib.ms_read_wait(self.h, C.byref(n), C.byref(t)), "ms_read_wait")
        return n.value, t.value

    def sync(self):
        self._check(self.lib.ms_sync(self.h), "ms_sync")

    def read_state(self, trips: bool = True) -> dict:
        s = ms_state(0, 0, 0)
        self.lib.ms_read_state(self.h, C.byref(s), 0)   # sizes only
        n = s.n_active
        out = dict(id=np.zeros(n, np.int32), lane=np.zeros(n, np.int32), route_idx=np.zeros(n, np.int32),
                   x=np.zeros(n, np.float32), v=np.zeros(n, np.float32))
        if trips:
            out["trip_status"] = np.zeros(self.n_trips, np.int32)
            out["t_arr"] = np.zeros(self.n_trips, np.int32)
        if getattr(self, "n_ctrl", 0) > 0:
            out["ctrl_state"] = np.zeros((self.n_ctrl, 3), np.int32)
        s = ms_state(n, 0, 0, *[_p(out.get(f)) for f in ("id", "lane", "route_idx", "x", "v", "trip_status", "t_arr",
                                                          "ctrl_state")])
        self._check(self.lib.ms_read_state(self.h, C.byref(s), 0), "ms_read_state")
        out["t"] = s.t
        out["n_active"] = s.n_active
        return out

    def read_state_device(self, x, v, lane, vid, route_idx=None) -> int:
        """Device-to-device copy into torch CUDA tensors of sufficient length; returns n."""
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        s = ms_state(_export_capacity(x, v, lane, vid, route_idx), 0, 0, ptr(vid), ptr(lane), ptr(route_idx),
                     ptr(x), ptr(v), None, None)
        self._check(self.lib.ms_read_state(self.h, C.byref(s), 1), "ms_read_state")
        return s.n_active

    def write_state(self, st: dict):
        n = int(st["id"].shape[0])
        keep = dict(id=np.ascontiguousarray(st["id"], np.int32), lane=np.ascontiguousarray(st["lane"], np.int32),
                    route_idx=np.ascontiguousarray(st["route_idx"], np.int32),
                    x=np.ascontiguousarray(st["x"], np.float32), v=np.ascontiguousarray(st["v"], np.float32),
                    t_arr=np.ascontiguousarray(st["t_arr"], np.int32))
        cs = st.get("ctrl_state")
        keep["ctrl_state"] = None if cs is None else np.ascontiguousarray(cs, np.int32).reshape(-1)
        s = ms_state(n, n, int(st["t"]), _p(keep["id"]), _p(keep["lane"]), _p(keep["route_idx"]),
                     _p(keep["x"]), _p(keep["v"]), None, _p(keep["t_arr"]), _p(keep["ctrl_state"]))
        self._check(self.lib.ms_write_state(self.h, C.byref(s)), "ms_write_state")

    def read_metrics(self, lanes: bool = True) -> dict:
        m = self.n_windows * self.n_lanes
        vs = np.zeros(m, np.float32) if lanes else None
        vc = np.zeros(m, np.int32) if lanes else None
        s = ms_metrics(_p(vs), _p(vc))
        self._check(self.lib.ms_read_metrics(self.h, C.byref(s)), "ms_read_metrics")
        out = dict(inserted=s.inserted, arrived=s.arrived, sum_tt=s.sum_travel_time, n_active=s.n_active,
                   t=s.t, movers=s.movers_last_step, err=s.err)
        if lanes:
            out["vsum"] = vs.reshape(self.n_windows, self.n_lanes)
            out["vcnt"] = vc.reshape(self.n_windows, self.n_lanes)
        return out

    def read_debug(self) -> dict:
        n = self.n_trips
        out = {f: np.full(n, -7, np.int32) for f in _DBG_I}
        out["active_before"][:] = 0
        out["inserted"][:] = 0
        out["flag"][:] = 0
        out.update({f: np.full(n, np.nan, np.float32) for f in _DBG_F})
        out["lc_learn"] = np.zeros(n, np.int32)
        out["lc_margin"] = np.full(n, np.nan, np.float32)
        out["lc_logit"] = np.full((n, 3), np.nan, np.float32)
        out["lc_feat"] = np.full((n, 16), np.nan, np.float32)
        s = ms_debug(*[_p(out[f]) for f in _DBG_I + _DBG_F + _DBG_LC])
        self._check(self.lib.ms_read_debug(self.h, C.byref(s)), "ms_read_debug")
        return out

    def set_lc_log(self, x=None, y=None, n=None):
        """Log (features, rule decision) of lane-change candidates into device tensors
        (x bf16 [cap,16], y int32 [cap], n int32 [1]); no arguments turns logging off."""
        given = [t is not None for t in (x, y, n)]
        if any(given) and not all(given):
            raise ValueError("set_lc_log takes x, y and n together, or none of them")
        cap = 0
        if all(given):
            import torch
            if (x.dtype != torch.bfloat16 or x.dim() != 2 or x.shape[1] != 16 or not x.is_contiguous()
                    or y.dtype != torch.int32 or not y.is_contiguous() or n.dtype != torch.int32 or n.numel() < 1):
                raise ValueError("set_lc_log: x bf16 [cap, 16], y int32 [cap], n int32 [1], contiguous")
            cap = min(int(y.numel()), int(x.shape[0]))
        self._check(self.lib.ms_set_lc_log(self.h, _dp(x), _dp(y), cap, _dp(n)), "ms_set_lc_log")

    def sample_trips(self, zone_edge, attract, gamma: int, n: int, t_span: int, seed: int):
        """Gravity OD sampling (GPU): returns (orig_edge, dest_edge, t_dep) int32 arrays."""
        z = np.ascontiguousarray(zone_edge, np.int32)
        a = np.ascontiguousarray(attract, np.float32)
        if a.shape != z.shape:
            raise ValueError("one attraction per zone")
        o = np.zeros(n, np.int32)
        d = np.zeros(n, np.int32)
        t = np.zeros(n, np.int32)
        self._check(self.lib.ms_sample_trips(self.h, int(z.shape[0]), _p(z), _p(a), int(gamma), int(n), int(t_span),
                                             int(seed) & 0xFFFFFFFFFFFFFFFF, _p(o), _p(d), _p(t)), "ms_sample_trips")
        return o, d, t

    def sample_trips_radiation(self, zone_edge, population, n: int, t_span: int, seed: int):
        """Radiation OD sampling (GPU): returns (orig_edge, dest_edge, t_dep) int32 arrays."""
        z = np.ascontiguousarray(zone_edge, np.int32)
        m = np.ascontiguousarray(population, np.float32)
        if m.shape != z.shape:
            raise ValueError("one population per zone")
        o = np.zeros(n, np.int32)
        d = np.zeros(n, np.int32)
        t = np.zeros(n, np.int32)
        self._check(self.lib.ms_sample_trips_radiation(self.h, int(z.shape[0]), _p(z), _p(m), int(n), int(t_span),
                                                       int(seed) & 0xFFFFFFFFFFFFFFFF, _p(o), _p(d), _p(t)),
                    "ms_sample_trips_radiation")
        return o, d, t

    def route_trips(self, orig, dest, capacity: int | None = None):
        """Least-cost lane-linked routes (GPU) for trips orig[i] -> dest[i] (edge ids):
        returns (route_off int64 [n+1], route_edges int32, n_unreachable)."""
        o = np.ascontiguousarray(orig, np.int32)
        d = np.ascontiguousarray(dest, np.int32)
        n = int(o.shape[0])
        off = np.zeros(n + 1, np.int64)
        cap = int(capacity) if capacity is not None else max(1, 64 * n)
        out = np.zeros(cap, np.int32)
        bad = C.c_int(0)
        rc = self.lib.ms_route_trips(self.h, n, _p(o), _p(d), _p(off), _p(out), cap, C.byref(bad))
        if rc == MS_ERR_CAPACITY:
            out = np.zeros(int(off[-1]), np.int32)
            rc = self.lib.ms_route_trips(self.h, n, _p(o), _p(d), _p(off), _p(out), int(off[-1]), C.byref(bad))
        self._check(rc, "ms_route_trips")
        return off, out[:int(off[-1])].copy(), int(bad.value)

    def set_lane_limits(self, lanes, vmax=None, closed=None):
        """Lane speed limits (m/s; <= 0 or inf: none) and closures for the given lanes, in
        effect from the next step."""
        ln = np.ascontiguousarray(lanes, np.int32)
        vm = None if vmax is None else np.ascontiguousarray(vmax, np.float32)
        cl = None if closed is None else np.ascontiguousarray(closed, np.int32)
        if (vm is not None and vm.shape != ln.shape) or (cl is not None and cl.shape != ln.shape):
            raise ValueError("one limit / closure flag per lane")
        self._check(self.lib.ms_set_lane_limits(self.h, int(ln.shape[0]), _p(ln), _p(vm), _p(cl)),
                    "ms_set_lane_limits")

    def set_lane_links(self, lanes, open_mask):
        """Dynamic lanes: bit j of open_mask[k] opens (1) or closes (0) the j-th lane link of
        edge lane lanes[k], in effect from the next step."""
        ln = np.ascontiguousarray(lanes, np.int32)
        mk = np.ascontiguousarray(open_mask, np.uint32)
        if ln.shape != mk.shape:
            raise ValueError("lanes and open_mask differ in length")
        self._check(self.lib.ms_set_lane_links(self.h, int(ln.shape[0]), _p(ln), _p(mk)), "ms_set_lane_links")

    def set_lc_model(self, params=None, margin: float = 0.2):
        """Use the learned lane-change decision (params: 5443 floats, host); None: rule."""
        a = None if params is None else np.ascontiguousarray(params, np.float32)
        if a is not None and a.size != MLP_NPARAM:
            raise ValueError(f"the model has {MLP_NPARAM} parameters")
        self._keep_model = a
        self._check(self.lib.ms_set_lc_model(self.h, _p(a), float(margin)), "ms_set_lc_model")

    def read_lc_stats(self) -> dict:
        out = np.zeros(12, np.int64)
        self._check(self.lib.ms_read_lc_stats(self.h, _p(out)), "ms_read_lc_stats")
        return dict(zip(LC_STAT_NAMES, out.tolist()))

    def test_withhold_copies(self, on: bool = True):
        """Steps that follow issue no bulk copy in the apply kernel (its waits run out and
        report MS_DEV_TIMEOUT); the state is invalid from then on."""
        self._check(self.lib.ms_test_withhold_copies(self.h, int(bool(on))), "ms_test_withhold_copies")

    def destroy(self):
        if self.h:
            self.lib.ms_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
