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


def _full_step_vs_oracle(sim, net, dem, label, theta=None, margin=0.2):
    """One production step of sim (already warmed up) against the oracle stepping from the
    GPU's own state over every vehicle; then the invariants of the state at that size and
    a checkpoint / resume.  theta: the learned lane-change model set on both sides."""
    st0 = sim.read_state()
    orc = oracle.Oracle(net, dem, P, n_windows=1, threads=os.cpu_count() or 1)
    if theta is not None:
        orc.set_lc_model(theta, margin)
    status, lane, x, v, rp, t_arr = parity.oracle_state_from_gpu(st0, orc.n)
    orc.set_state(status, lane, x, v, rp, st0["t"], t_arr)
    sim.step(1)
    sim.sync()
    gs = sim.read_state()
    m = sim.read_metrics(lanes=False)
    assert m["err"] == 0
    lc_stats = sim.read_lc_stats() if theta is not None else None
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
    print(label, "active", int(act.sum()), "flagged", n_flag, "compared", still.size)
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
    return od, os_, act, ok, lc_stats


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
    _full_step_vs_oracle(sim, net, dem, workload)


@pytest.fixture(scope="module")
def small_trained():
    """A lane-change network trained by the library's kernels on about 2M decisions logged
    from the small grid's mixed scenarios (the benchmark trains on 50M; parity does not
    depend on how well the network agrees with the rule)."""
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2405_12520_b300 import learned
    x, y, _ = learned.collect_batched(learned.mixed_specs(512), P, 3600, 2_000_000)
    cw, _ = learned.class_weights(y)
    theta, _ = learned.train(x, y, epochs=2, batch=8192, lr=2e-3, seed=1, class_w=cw)
    return theta


@pytest.mark.parametrize("workload", ["learned1m", "learned5m"])
def test_full_size_learned_step_matches_oracle(small_trained, workload):
    """The learned form at the sizes the learned benchmark times (the 1M-vehicle grid with
    inflow; 5M vehicles near jam density on the same grid), in its launch configuration
    (the learned decide instance listing candidates, k_learn, the step's graph): one step
    after the warm-up against the oracle's learned step (R19) over every vehicle, with
    decisions flagged where R19's flag rule says a rounding could change them."""
    sys.path.insert(0, ROOT)
    import bench
    if workload == "learned5m":
        net = synth.large_grid_network()
        dem = synth.place_vehicles(net, 5_000_000, seed=3, min_spacing=6.0)
    else:
        net, dem, _ = bench.workload("grid1m", 3)
    theta = small_trained
    sim = moss.Sim(P, n_windows=1)
    sim.load_network(net)
    sim.add_vehicles(dem)
    sim.set_lc_model(theta, 0.2)
    sim.step(10)
    sim.sync()
    sim.set_lc_model(theta, 0.2)              # counters of the compared step only
    od, os_, act, ok, st = _full_step_vs_oracle(sim, net, dem, workload, theta=theta)
    learned_by_oracle = (od["lc_learn"] == 1) & act
    n_learn = int(learned_by_oracle.sum())
    n_net = int((learned_by_oracle & (od["lc_margin"] >= 0.2)).sum())   # the network's own class
    print(workload, "learned candidates", n_learn, "decided by the network", n_net,
          "unflagged", int((learned_by_oracle & ok).sum()))
    # near jam density few vehicles have room to change (61 candidates in this step at 5M)
    assert n_learn > (1000 if workload == "learned1m" else 30) and n_net > 0.9 * n_learn
    # the GPU listed the oracle's candidates (up to flagged safety decisions)
    assert abs(st["candidates"] - n_learn) <= 0.01 * n_learn + 10


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
