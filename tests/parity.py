"""Helpers that run the CUDA path and the oracle from the same state and compare them.

Tolerances (single step from identical FP32 states):
  - integers (neighbour ids, lane, route index, status, lane-change decision, departures):
    bit-exact for every vehicle whose decisions were not flagged by either side;
  - |Δa| <= 1e-4 m/s^2 (after the [a_min, a_max] clamp), |Δv| <= 1e-4 m/s,
    |Δx| <= max(1e-4, 2 ulp_fp32(x)) m;
  - a vehicle is flagged when a decision margin (MOBIL incentive - threshold, a~_n + b_safe,
    follower guard, new-leader gap, yellow stop test, x' - len, look-ahead horizon, merge
    distance tie, lane-change zones, departure room) lies within 1e-3 of its threshold on
    either side; flagged vehicles are counted and reported, not compared.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2405_12520_b300 import moss

A_TOL = 1e-4
V_TOL = 1e-4
X_TOL = 1e-4


def x_tol(x):
    x = np.abs(np.asarray(x, np.float64))
    return np.maximum(X_TOL, 2.0 * np.spacing(x.astype(np.float32)).astype(np.float64))


def gpu_sim(net, dem, params, debug=True, n_windows=1, block=0):
    s = moss.Sim(params, debug=debug, n_windows=n_windows, block=block)
    s.load_network(net)
    s.add_vehicles(dem)
    return s


def oracle_state_from_gpu(st: dict, n_trips: int):
    """GPU read_state -> per-trip arrays for Oracle.set_state."""
    status = st["trip_status"].copy()
    lane = np.zeros(n_trips, np.int32)
    x = np.zeros(n_trips)
    v = np.zeros(n_trips)
    rp = np.zeros(n_trips, np.int32)
    lane[st["id"]] = st["lane"]
    x[st["id"]] = st["x"].astype(np.float64)
    v[st["id"]] = st["v"].astype(np.float64)
    rp[st["id"]] = st["route_idx"]
    return status, lane, x, v, rp, st["t_arr"].copy()


def step_pair(sim: moss.Sim, orc: oracle.Oracle):
    """Load the GPU's current state into the oracle, step both once, return records."""
    st0 = sim.read_state()
    status, lane, x, v, rp, t_arr = oracle_state_from_gpu(st0, orc.n)
    orc.set_state(status, lane, x, v, rp, st0["t"], t_arr)
    if "ctrl_state" in st0:   # max-pressure controllers (identical in fixed-time mode)
        orc.set_ctrl_state(st0["ctrl_state"])
    sim.step(1)
    sim.sync()
    gd = sim.read_debug()
    gs = sim.read_state()
    _, od = orc.step(debug=True)
    os_ = orc.state()
    if "ctrl_state" in gs:
        os_["ctrl_state"] = orc.ctrl_state()
    return st0, gd, gs, od, os_


def compare_step(gd, gs, od, os_, n_trips, report=None, max_flag_frac=0.05):
    """Assert parity of one step; returns a dict of counts."""
    if "ctrl_state" in gs and "ctrl_state" in os_:   # controllers advanced to the next step
        assert np.array_equal(gs["ctrl_state"], os_["ctrl_state"]), "controller states differ"
    act = od["active_before"] == 1
    assert np.array_equal(act, gd["active_before"] == 1), "different active sets"
    flagged = (od["flag"] == 1) | (gd["flag"] == 1)
    cmp = act & ~flagged
    ids = np.nonzero(cmp)[0]
    for f in ("lead_kind", "lead_id", "lc_cand", "lc_dir", "tau_lead", "tau_foll", "old_foll"):
        g, o = gd[f][ids], od[f][ids]
        bad = np.nonzero(g != o)[0]
        assert bad.size == 0, f"{f} differs for ids {ids[bad[:10]].tolist()}: gpu {g[bad[:10]].tolist()} oracle {o[bad[:10]].tolist()}"
    for f in ("a_own", "a_use"):
        d = np.abs(gd[f][ids].astype(np.float64) - od[f][ids])
        assert d.size == 0 or d.max() <= A_TOL, f"{f} max diff {d.max()} at id {ids[np.argmax(d)]}"
    veh = ids[od["lead_kind"][ids] != 0]
    d = np.abs(gd["s_own"][veh].astype(np.float64) - od["s_own"][veh])
    assert d.size == 0 or d.max() <= 1e-3, f"s_own max diff {d.max()}"
    # new state by trip id
    g_status = gs["trip_status"]
    o_status = os_["status"]
    g_ins = gd["inserted"] == 1
    o_ins = od["inserted"] == 1
    ins_ok = ~flagged
    assert np.array_equal(g_ins[ins_ok], o_ins[ins_ok]), "departures differ"
    both = np.nonzero((cmp | (g_ins & o_ins)))[0]
    assert np.array_equal(g_status[both], o_status[both]), "status differs"
    still = both[o_status[both] == 1]
    g_lane = np.full(n_trips, -1, np.int64)
    g_x = np.full(n_trips, np.nan)
    g_v = np.full(n_trips, np.nan)
    g_rp = np.full(n_trips, -1, np.int64)
    g_lane[gs["id"]] = gs["lane"]
    g_x[gs["id"]] = gs["x"]
    g_v[gs["id"]] = gs["v"]
    g_rp[gs["id"]] = gs["route_idx"]
    bad = still[g_lane[still] != os_["lane"][still]]
    assert bad.size == 0, f"lane differs for ids {bad[:10].tolist()}"
    assert np.array_equal(g_rp[still], os_["rp"][still]), "route index differs"
    dx = np.abs(g_x[still] - os_["x"][still])
    tol = x_tol(os_["x"][still])
    assert dx.size == 0 or np.all(dx <= tol), f"x max excess {np.max(dx - tol)} at id {still[np.argmax(dx - tol)]}"
    dv = np.abs(g_v[still] - os_["v"][still])
    assert dv.size == 0 or dv.max() <= V_TOL, f"v max diff {dv.max()} at id {still[np.argmax(dv)]}"
    # the GPU state is sorted by (lane, x)
    gl, gx = gs["lane"].astype(np.int64), gs["x"]
    assert np.all((gl[1:] > gl[:-1]) | ((gl[1:] == gl[:-1]) & (gx[1:] >= gx[:-1]))), "GPU state not sorted"
    n_act = int(act.sum())
    n_flag = int((act & flagged).sum())
    if n_act:
        assert n_flag <= max_flag_frac * n_act + 2, f"{n_flag} of {n_act} flagged"
    out = dict(active=n_act, flagged=n_flag, compared=int(ids.size),
               changes=int((gd["lc_dir"][ids] != 0).sum()),
               moved_on=int(still.size), inserted=int(g_ins.sum()))
    if report is not None:
        report.append(out)
    return out



# absolute part of the oracle's bound on the FP32 path's error in each learned input (R19):
# gaps and the distance to the lane end (FP32 gaps within 1e-3 m, scaled by 1/100), and
# accelerations (within 1e-4 m/s^2, scaled by 1/a_max); speeds carry FP32 rounding only
IN_ABS = np.zeros(16)
IN_ABS[[2, 6, 8, 13, 15]] = 1e-5
IN_ABS[[4, 10, 11]] = 5e-5


def near_bf16_boundary(f, delta):
    """Whether each value of f lies within delta of a BF16 rounding boundary."""
    from oracle import mlp
    r = mlp.bf16(f)
    a = np.abs(r)
    _, e = np.frexp(np.where(a > 0, a, 1.0))
    ulp = np.ldexp(1.0, e - 8)
    ulp_in = np.where(a == np.ldexp(1.0, e - 1), ulp / 2, ulp)
    d = np.minimum(np.abs(np.abs(f) - (a + ulp / 2)), np.abs(np.abs(f) - (a - ulp_in / 2)))
    return (a > 0) & (d <= delta)


def compare_learned(gd, od, theta, report=None):
    """Parity of the learned lane-change decisions of one step (reading R19), after
    compare_step has checked the decisions themselves (lc_dir) of every unflagged vehicle.
    For every unflagged vehicle:
      - the network decided on both sides or on neither;
      - its 16 BF16 inputs equal the oracle's inputs rounded to BF16, except an input whose
        oracle value lies within the FP32 path's error of a BF16 rounding boundary (there:
        within one BF16 step plus that error);
      - its logits agree within the FP32 accumulation bound of the last layer plus the
        summed logit changes of rounding, one at a time, each input or hidden value near a
        BF16 rounding boundary the other way (oracle/mlp.flip_sensitivity), plus 1e-6.
    Returns counts."""
    from oracle import mlp
    act = od["active_before"] == 1
    flagged = (od["flag"] == 1) | (gd["flag"] == 1)
    cmp = act & ~flagged
    bad = np.nonzero(cmp & ((gd["lc_learn"] == 1) != (od["lc_learn"] == 1)))[0]
    assert bad.size == 0, f"learned sets differ for ids {bad[:10].tolist()}"
    L = np.nonzero(cmp & (od["lc_learn"] == 1))[0]
    fo, fg = od["lc_feat"][L], gd["lc_feat"][L].astype(np.float64)
    fb = mlp.bf16(fo)
    nin = near_bf16_boundary(fo, 2.0 ** -22 * np.abs(fo) + IN_ABS)
    bad = np.nonzero(np.any((fg != fb) & ~nin, axis=1))[0]
    assert bad.size == 0, f"BF16 inputs differ for ids {L[bad[:5]].tolist()}: gpu {fg[bad[:1]]} oracle {fb[bad[:1]]}"
    # near a boundary the FP32 value itself may differ from the FP64 one by up to delta (R19),
    # and then round the other way: one BF16 step of the value plus delta (near zero, where a
    # BF16 step is tiny, delta dominates)
    step = 2.0 ** -7 * np.abs(fo) + 2.0 ** -22 * np.abs(fo) + IN_ABS
    over = np.argwhere(nin & (np.abs(fg - fo) > step))
    assert over.size == 0, ("an input off by more than one BF16 step and its FP32 error: (candidate id, "
                            "input, gpu, oracle) "
                            + str([(int(L[r]), int(q), float(fg[r, q]), float(fo[r, q])) for r, q in over[:5]]))
    zo, zg = od["lc_logit"][L], gd["lc_logit"][L].astype(np.float64)
    z, _, _, zbound, _, _ = mlp.flip_sensitivity(np.asarray(theta, np.float64), fo, 0.0,
                                                 in_delta=2.0 ** -22 * np.abs(fo) + IN_ABS)
    assert np.allclose(z, zo, rtol=1e-12, atol=1e-12), "oracle logits differ from oracle/mlp"
    dz = np.abs(zg - zo)
    over = dz - (zbound + 1e-6)
    assert dz.size == 0 or over.max() <= 0, f"logit excess {over.max()} at id {L[np.argmax(over.max(axis=1))]}"
    ex = np.nonzero(od["lc_near"][L] == 0)[0]
    out = dict(learned=int(L.size), exact=int(ex.size), near_inputs=int(nin.any(axis=1).sum()),
               learned_flagged=int((act & flagged & ((od["lc_learn"] == 1) | (gd["lc_learn"] == 1))).sum()),
               changes=int((od["lc_dir"][L] != 0).sum()), max_dz=float(dz.max()) if dz.size else 0.0)
    if report is not None:
        report.append(out)
    return out
