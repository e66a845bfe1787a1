"""Parity at the benchmark's full sizes, in the launch configuration bench.py times (the
production decide instance, default launch shapes, the step's CUDA graph): one step from the
GPU's own state after the benchmark's warm-up, against the FP64 oracle stepping from the
same state, over every vehicle; plus the invariants of the state at that size."""
import os
import sys

import numpy as np
import pytest

import oracle
import parity
from paper_2405_12520_b300 import moss, synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = synth.default_params()


@pytest.mark.parametrize("workload", ["grid1m", "city5m"])
def test_full_size_step_matches_oracle(workload):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sys.path.insert(0, ROOT)
    import bench
    net, dem, _ = bench.workload(workload, 3)
    sim = moss.Sim(P, n_windows=1)           # bench.py's configuration (block 0: default shapes)
    sim.load_network(net)
    sim.add_vehicles(dem)
    sim.step(10)                              # the benchmark's warm-up
    st0 = sim.read_state()
    orc = oracle.Oracle(net, dem, P, n_windows=1)
    status, lane, x, v, rp, t_arr = parity.oracle_state_from_gpu(st0, orc.n)
    orc.set_state(status, lane, x, v, rp, st0["t"], t_arr)
    sim.step(1)
    sim.sync()
    gs = sim.read_state()
    m = sim.read_metrics(lanes=False)
    assert m["err"] == 0
    err, od = orc.step(debug=True)
    assert err == 0
    os_ = orc.state()
    n = orc.n
    act = od["active_before"] == 1
    assert int(act.sum()) == st0["n_active"]
    flagged = od["flag"] == 1
    # trips the oracle did not flag: status, lane, route index bit-exact; x, v within tolerance
    ok = ~flagged & ((act) | (od["inserted"] == 1))
    np.testing.assert_array_equal(gs["trip_status"][ok], os_["status"][ok])
    still = np.nonzero(ok & (os_["status"] == 1))[0]
    g_lane = np.full(n, -1, np.int64)
    g_x = np.full(n, np.nan)
    g_v = np.full(n, np.nan)
    g_rp = np.full(n, -1, np.int64)
    g_lane[gs["id"]] = gs["lane"]
    g_x[gs["id"]] = gs["x"]
    g_v[gs["id"]] = gs["v"]
    g_rp[gs["id"]] = gs["route_idx"]
    bad = still[g_lane[still] != os_["lane"][still]]
    assert bad.size == 0, f"lane differs for {bad.size} trips, e.g. {bad[:10].tolist()}"
    np.testing.assert_array_equal(g_rp[still], os_["rp"][still])
    dx = np.abs(g_x[still] - os_["x"][still])
    assert np.all(dx <= parity.x_tol(os_["x"][still])), f"x max diff {dx.max()}"
    dv = np.abs(g_v[still] - os_["v"][still])
    assert dv.max() <= parity.V_TOL, f"v max diff {dv.max()}"
    n_flag = int((act & flagged).sum())
    print(workload, "active", int(act.sum()), "flagged", n_flag, "compared", still.size)
    assert n_flag <= 0.05 * int(act.sum())
    # invariants at full size: sorted by (lane, x), gap >= 0 up to FP32 rounding, every trip
    # waiting, active or arrived exactly once
    gl, gx = gs["lane"].astype(np.int64), gs["x"].astype(np.float64)
    same = gl[1:] == gl[:-1]
    assert np.all((gl[1:] > gl[:-1]) | (same & (gx[1:] >= gx[:-1])))
    gap = (gx[1:] - gx[:-1])[same] - P["veh_len"]
    ulp = np.spacing(gs["x"][1:][same].astype(np.float32)).astype(np.float64)
    assert np.all(gap >= -2.0 * ulp - 1e-6), gap.min()
    counts = np.bincount(gs["trip_status"], minlength=3)
    assert counts[1] == gs["n_active"] and counts.sum() == n
    assert len(np.unique(gs["id"])) == gs["n_active"]
    # checkpoint / resume at this size: the read state loads back and steps on
    sim.write_state(gs)
    sim.step(1)
    sim.sync()
    assert sim.read_metrics(lanes=False)["err"] == 0


def test_full_size_batch_step_matches_oracle():
    """The 256-scenario batch (4.78M vehicles, 4.96M lanes) as bench.py runs it (batch
    loaders, autotuned launch shapes, graph steps): one step after the warm-up against the
    oracle on the union network, over every vehicle."""
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sc = synth.batch_scenarios(256, seed=3, n_lanes=3, link_len=300.0)
    nets, dems = [n for n, _ in sc], [d for _, d in sc]
    b = moss.Sim(P)
    b.load_network_batch(nets)
    b.add_vehicles_batch(dems)
    b.autotune(trial_steps=3)
    b.step(5)
    st0 = b.read_state()
    unet, udem = synth.union(nets, dems)
    orc = oracle.Oracle(unet, udem, P)
    status, lane, x, v, rp, t_arr = parity.oracle_state_from_gpu(st0, orc.n)
    orc.set_state(status, lane, x, v, rp, st0["t"], t_arr)
    b.step(1)
    b.sync()
    gs = b.read_state()
    assert b.read_metrics(lanes=False)["err"] == 0
    err, od = orc.step(debug=True)
    assert err == 0
    os_ = orc.state()
    act = od["active_before"] == 1
    ok = (od["flag"] == 0) & (act | (od["inserted"] == 1))
    np.testing.assert_array_equal(gs["trip_status"][ok], os_["status"][ok])
    still = np.nonzero(ok & (os_["status"] == 1))[0]
    n = orc.n
    g_lane = np.full(n, -1, np.int64)
    g_x = np.full(n, np.nan)
    g_v = np.full(n, np.nan)
    g_lane[gs["id"]] = gs["lane"]
    g_x[gs["id"]] = gs["x"]
    g_v[gs["id"]] = gs["v"]
    assert np.array_equal(g_lane[still], os_["lane"][still])
    assert np.all(np.abs(g_x[still] - os_["x"][still]) <= parity.x_tol(os_["x"][still]))
    assert np.abs(g_v[still] - os_["v"][still]).max() <= parity.V_TOL
    print("batch256 active", int(act.sum()), "compared", still.size)
    assert still.size > 0.95 * int(act.sum())


def test_full_size_long_run_keeps_invariants():
    """grid1m for 1200 steps (departures, arrivals, signals, four five-minute windows): no
    device error bit, the state sorted with gaps >= 0 up to FP32 rounding, every trip
    counted once, and the lane metrics' counts equal to the active vehicles summed over the
    steps."""
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sys.path.insert(0, ROOT)
    import bench
    net, dem, _ = bench.workload("grid1m", 3)
    sim = moss.Sim(P, n_windows=4)
    sim.load_network(net)
    sim.add_vehicles(dem)
    active_sum = 0
    for _ in range(1200):   # the snapshot of every step is counted once in the lane metrics
        active_sum += sim.read_metrics(lanes=False)["n_active"]
        sim.step(1)
    sim.sync()
    m = sim.read_metrics()
    assert int(m["vcnt"].sum()) == active_sum
    assert m["err"] == 0
    gs = sim.read_state()
    gl, gx = gs["lane"].astype(np.int64), gs["x"].astype(np.float64)
    same = gl[1:] == gl[:-1]
    assert np.all((gl[1:] > gl[:-1]) | (same & (gx[1:] >= gx[:-1])))
    gap = (gx[1:] - gx[:-1])[same] - P["veh_len"]
    ulp = np.spacing(gs["x"][1:][same].astype(np.float32)).astype(np.float64)
    assert np.all(gap >= -2.0 * ulp - 1e-6)
    counts = np.bincount(gs["trip_status"], minlength=3)
    assert counts[1] == gs["n_active"] and counts.sum() == dem.n
    assert counts[2] == m["arrived"] and m["inserted"] > 0
    assert m["vcnt"].sum() > 0 and np.all(m["vsum"] >= 0)
