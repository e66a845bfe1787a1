"""CUDA path vs the FP64 oracle, through the C ABI (libmoss103.so via the ctypes binding).

Single steps start from identical FP32 states (the GPU state is loaded into the oracle);
tolerances are documented in tests/parity.py."""
import numpy as np
import pytest

import oracle
import parity
import netkit
from paper_2405_12520_b300 import synth

pytestmark = pytest.mark.gpu
P = synth.default_params()


def _need_gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _net(kind):
    if kind == "grid4x2":
        return synth.grid_network(4, 4, 2, 200.0, 30, 3, "zero")
    if kind == "grid12x3":   # ~6.6k lanes: several lane-scan tiles
        return synth.grid_network(12, 12, 3, 200.0, 30, 3, "wave")
    if kind == "delaunay":
        return synth.delaunay_network(120, box=3000.0, seed=7)
    raise ValueError(kind)


CASES = [
    # network, placed vehicles, waiting trips, spacing, internal fraction, t0, p_lc
    ("grid4x2", 300, 200, 5.6, 0.4, 0, 1.0),
    ("grid4x2", 300, 200, 9.0, 0.4, 31, 0.5),
    ("grid12x3", 5003, 800, 7.0, 0.3, 64, 1.0),
    ("grid12x3", 9001, 0, 5.4, 0.5, 1001, 1.0),
    ("delaunay", 2500, 500, 6.0, 0.5, 3, 1.0),
    ("delaunay", 3001, 300, 9.0, 0.2, 66, 0.5),
]


@pytest.mark.parametrize("kind,n_place,n_wait,spacing,ifrac,t0,p_lc", CASES)
def test_single_steps_match_oracle(kind, n_place, n_wait, spacing, ifrac, t0, p_lc):
    _need_gpu()
    net = _net(kind)
    dem = synth.place_vehicles(net, n_place, seed=11 + t0, min_spacing=spacing, internal_frac=ifrac)
    if n_wait:
        dem = synth.merge_demands(dem, synth.uniform_trips(net, n_wait, 40, seed=5 + t0))
    params = dict(P, p_lc=p_lc, seed=1234 + t0)
    sim = parity.gpu_sim(net, dem, params)
    st = sim.read_state()
    st["t"] = t0
    sim.write_state(st)
    orc = oracle.Oracle(net, dem, params)
    rep = []
    for k in range(8):
        _, gd, gs, od, os_ = parity.step_pair(sim, orc)
        parity.compare_step(gd, gs, od, os_, dem.n, report=rep)
    tot = {k: sum(r[k] for r in rep) for k in rep[0]}
    print(kind, tot)
    assert tot["compared"] > 0.9 * tot["active"]
    assert tot["changes"] > 0 or p_lc < 1.0


@pytest.mark.parametrize("kind,t0", [("grid12x3", 64), ("delaunay", 3)])
def test_single_steps_match_oracle_threshold_jitter(kind, t0):
    """The randomized-MOBIL variant with per-trip threshold jitter (R12)."""
    _need_gpu()
    net = _net(kind)
    dem = synth.place_vehicles(net, 5003 if kind == "grid12x3" else 2500, seed=17 + t0, min_spacing=7.0,
                               internal_frac=0.3)
    params = dict(P, mobil_th_jitter=0.6, seed=99 + t0)
    sim = parity.gpu_sim(net, dem, params)
    st = sim.read_state()
    st["t"] = t0
    sim.write_state(st)
    orc = oracle.Oracle(net, dem, params)
    rep = []
    for k in range(8):
        _, gd, gs, od, os_ = parity.step_pair(sim, orc)
        parity.compare_step(gd, gs, od, os_, dem.n, report=rep)
    tot = {k: sum(r[k] for r in rep) for k in rep[0]}
    print(kind, tot)
    assert tot["compared"] > 0.9 * tot["active"]
    assert tot["changes"] > 0


MP = dict(P, signal_mode=1, mp_interval=10)


@pytest.mark.parametrize("kind,t0", [("grid12x3", 57), ("delaunay", 66)])
def test_single_steps_match_oracle_max_pressure(kind, t0):
    """Max-pressure signals (R13): decisions at steps 60 / 70 fall inside the 8 compared
    steps; the controllers' state is compared after every step."""
    _need_gpu()
    net = _net(kind)
    dem = synth.merge_demands(synth.place_vehicles(net, 5003 if kind == "grid12x3" else 2500, seed=31 + t0,
                                                   min_spacing=7.0, internal_frac=0.3),
                              synth.uniform_trips(net, 400, 40, seed=32 + t0))
    params = dict(MP, seed=7 + t0)
    sim = parity.gpu_sim(net, dem, params)
    st = sim.read_state()
    st["t"] = t0
    sim.write_state(st)
    orc = oracle.Oracle(net, dem, params)
    rep = []
    for k in range(8):
        _, gd, gs, od, os_ = parity.step_pair(sim, orc)
        parity.compare_step(gd, gs, od, os_, dem.n, report=rep)
    tot = {k: sum(r[k] for r in rep) for k in rep[0]}
    print(kind, tot, "pending", int((gs["ctrl_state"][:, 1] >= 0).sum()))
    assert tot["compared"] > 0.9 * tot["active"]


def test_lockstep_small_grid_max_pressure():
    _need_gpu()
    net, dem = synth.small_grid_workload(3)
    sim = parity.gpu_sim(net, dem, MP, n_windows=12)
    orc = oracle.Oracle(net, dem, MP, n_windows=12)
    rep = []
    for t in range(1500):
        if t % 5 == 0:
            _, gd, gs, od, os_ = parity.step_pair(sim, orc)
            parity.compare_step(gd, gs, od, os_, dem.n, report=rep)
        else:
            sim.step(1)
    sim.sync()
    assert sim.read_metrics(lanes=False)["err"] == 0
    tot = {k: sum(r[k] for r in rep) for k in rep[0]}
    print(tot)
    assert tot["flagged"] <= 0.01 * tot["active"]


def test_resume_is_bit_exact_max_pressure():
    _need_gpu()
    net, dem = synth.small_grid_workload(2)
    a = parity.gpu_sim(net, dem, MP, debug=False)
    a.step(705)
    sa = a.read_state()
    b = parity.gpu_sim(net, dem, MP, debug=False)
    b.step(303)
    mid = b.read_state()
    c = parity.gpu_sim(net, dem, MP, debug=False)
    c.write_state(mid)   # vehicles and controllers
    c.step(402)
    sc = c.read_state()
    for k in ("id", "lane", "x", "v", "route_idx", "t_arr", "t", "ctrl_state"):
        np.testing.assert_array_equal(sa[k], sc[k])


@pytest.mark.parametrize("kind,t0", [("grid12x3", 12), ("delaunay", 5)])
def test_single_steps_match_oracle_lane_limits(kind, t0):
    """Lane speed limits on 15% of the lanes (U[5, 12] m/s) and 3% of the lanes closed (R14),
    set through the modification call on both sides."""
    _need_gpu()
    net = _net(kind)
    dem = synth.merge_demands(synth.place_vehicles(net, 5003 if kind == "grid12x3" else 2500, seed=41 + t0,
                                                   min_spacing=7.0, internal_frac=0.3),
                              synth.uniform_trips(net, 400, 40, seed=42 + t0))
    rng = np.random.default_rng(43 + t0)
    lim = np.nonzero(rng.random(net.n_lanes) < 0.15)[0]
    shut = np.nonzero(rng.random(net.n_lanes) < 0.03)[0]
    vmax = rng.uniform(5.0, 12.0, lim.size).astype(np.float32)
    sim = parity.gpu_sim(net, dem, P)
    st = sim.read_state()
    st["t"] = t0
    sim.write_state(st)
    orc = oracle.Oracle(net, dem, P)
    for side in (sim, orc):
        side.set_lane_limits(lim, vmax=vmax)
        side.set_lane_limits(shut, closed=np.ones(shut.size, np.int32))
    rep = []
    for k in range(8):
        _, gd, gs, od, os_ = parity.step_pair(sim, orc)
        parity.compare_step(gd, gs, od, os_, dem.n, report=rep)
    tot = {k: sum(r[k] for r in rep) for k in rep[0]}
    print(kind, tot)
    assert tot["compared"] > 0.9 * tot["active"]
    # lifting every modification returns to the plain instance: same as never setting them
    sim.set_lane_limits(lim, vmax=np.zeros(lim.size, np.float32))
    sim.set_lane_limits(shut, closed=np.zeros(shut.size, np.int32))
    ref = parity.gpu_sim(net, dem, P, debug=False)
    cur = sim.read_state()
    ref.write_state(cur)
    sim.step(5)
    ref.step(5)
    a, b = sim.read_state(), ref.read_state()
    for k in ("id", "lane", "x", "v", "route_idx"):
        np.testing.assert_array_equal(a[k], b[k])


def test_single_steps_match_oracle_extreme_states():
    """Short links (25 m edges, 21+ m junction lanes) with a 500 m look-ahead, so the
    12-lane hop cap ends searches; vehicles standing exactly at lane ends and bumper to
    bumper (gap 0, v = 0) queues; plus moving vehicles.  Parity over 8 steps."""
    _need_gpu()
    net = synth.grid_network(6, 6, 2, 25.0, 30, 3, "random", seed=4)
    rng = np.random.default_rng(12)
    lanes, xs, vs, routes = [], [], [], []
    edge_lanes = np.nonzero(net.lane_edge >= 0)[0]
    for l in rng.choice(edge_lanes, 40, replace=False):
        e = int(net.lane_edge[l])
        # a next edge this lane links to (its first link's exit edge)
        k = int(net.succ_off[l])
        nxt = int(net.succ_edge[k])
        L = float(net.lane_len[l])
        kind = rng.integers(0, 3)
        if kind == 0:     # standing at the lane end
            pos, spd = [L], [0.0]
        elif kind == 1:   # bumper-to-bumper standstill queue ending at the lane end
            pos, spd = [L - 5.0 * q for q in range(4)][::-1], [0.0] * 4
        else:             # two moving vehicles
            pos, spd = [3.0, 14.0], [float(rng.uniform(3, 12)), float(rng.uniform(3, 12))]
        for x, v in zip(pos, spd):
            lanes.append(int(l))
            xs.append(x)
            vs.append(v)
            routes.append([e, nxt])
    dem = netkit.vehicles(lanes, xs, vs, routes)
    params = dict(P, d_look=500.0)
    sim = parity.gpu_sim(net, dem, params)
    orc = oracle.Oracle(net, dem, params)
    rep = []
    for k in range(8):
        _, gd, gs, od, os_ = parity.step_pair(sim, orc)
        # vehicles standing exactly at a lane end or at gap 0 sit exactly on decision
        # thresholds (margin 0), so many are flagged by design; the rest must match
        parity.compare_step(gd, gs, od, os_, dem.n, report=rep, max_flag_frac=0.5)
    tot = {k: sum(r[k] for r in rep) for k in rep[0]}
    print(tot)
    assert tot["compared"] > 0.5 * tot["active"]
    assert sim.read_metrics(lanes=False)["err"] == 0


def test_lockstep_small_grid_full_run():
    """The small grid workload run on the GPU for 3600 steps; every 5th step the oracle
    repeats the GPU's step from the GPU's state."""
    _need_gpu()
    net, dem = synth.small_grid_workload(1)
    sim = parity.gpu_sim(net, dem, P, n_windows=12)
    orc = oracle.Oracle(net, dem, P, n_windows=12)
    rep = []
    for t in range(3600):
        if t % 5 == 0:
            _, gd, gs, od, os_ = parity.step_pair(sim, orc)
            parity.compare_step(gd, gs, od, os_, dem.n, report=rep)
        else:
            sim.step(1)
    sim.sync()
    m = sim.read_metrics(lanes=False)
    assert m["err"] == 0
    st = sim.read_state()
    assert st["n_active"] == 0 and m["arrived"] == dem.n
    tot = {k: sum(r[k] for r in rep) for k in rep[0]}
    print(tot)
    assert tot["flagged"] <= 0.01 * tot["active"]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_whole_run_statistics_small_grid(seed):
    """Free-running 3600-step runs (FP32 GPU vs FP64 oracle diverge microscopically):
    completed trips and per-window network mean speed within 2%; per-lane 5-minute mean
    speeds within 2% on average over lanes with at least 300 vehicle-steps."""
    _need_gpu()
    net, dem = synth.small_grid_workload(seed)
    sim = parity.gpu_sim(net, dem, P, debug=False, n_windows=12)
    sim.step(3600)
    sim.sync()
    gm = sim.read_metrics()
    orc = oracle.Oracle(net, dem, P, n_windows=12)
    orc.run(3600)
    om = orc.metrics()
    assert abs(gm["arrived"] - om["arrived"]) <= 0.02 * om["arrived"]
    assert abs(gm["sum_tt"] / gm["arrived"] - om["sum_tt"] / om["arrived"]) <= 0.02 * om["sum_tt"] / om["arrived"]
    gv, gc = gm["vsum"].astype(np.float64), gm["vcnt"].astype(np.float64)
    ov, oc = om["vsum"], om["vcnt"].astype(np.float64)
    w = (oc.sum(1) > 0) & (gc.sum(1) > 0)
    net_g = gv.sum(1)[w] / gc.sum(1)[w]
    net_o = ov.sum(1)[w] / oc.sum(1)[w]
    busy = oc.sum(1)[w] >= 2000
    assert np.all(np.abs(net_g - net_o)[busy] <= 0.02 * net_o[busy]), (net_g, net_o)
    m = (gc >= 300) & (oc >= 300)
    rel = np.abs(gv[m] / gc[m] - ov[m] / oc[m]) / (ov[m] / oc[m])
    print("lanes compared", m.sum(), "mean rel", rel.mean(), "p90", np.quantile(rel, 0.9))
    assert rel.mean() <= 0.02


def test_run_invariants_and_determinism_delaunay():
    _need_gpu()
    net = synth.delaunay_network(150, box=3500.0, seed=9)
    dem = synth.merge_demands(synth.place_vehicles(net, 3000, seed=9, min_spacing=6.0, internal_frac=0.5),
                              synth.uniform_trips(net, 2000, 600, seed=10))
    a = parity.gpu_sim(net, dem, P)          # debug: device order/gap check every step
    a.step(500)
    a.sync()
    ma = a.read_metrics(lanes=False)
    assert ma["err"] == 0
    sa = a.read_state()
    placed = int((dem.lane >= 0).sum())
    assert ma["inserted"] + placed == sa["n_active"] + ma["arrived"]
    b = parity.gpu_sim(net, dem, P, debug=False)
    b.step(500)
    sb = b.read_state()
    for k in ("id", "lane", "x", "v", "route_idx", "t_arr"):
        np.testing.assert_array_equal(sa[k], sb[k])


def test_resume_is_bit_exact():
    _need_gpu()
    net, dem = synth.small_grid_workload(2)
    a = parity.gpu_sim(net, dem, P, debug=False)
    a.step(700)
    sa = a.read_state()
    b = parity.gpu_sim(net, dem, P, debug=False)
    b.step(300)
    mid = b.read_state()
    c = parity.gpu_sim(net, dem, P, debug=False)
    c.write_state(mid)
    c.step(400)
    sc = c.read_state()
    for k in ("id", "lane", "x", "v", "route_idx", "t_arr", "t"):
        np.testing.assert_array_equal(sa[k], sc[k])


def test_edge_cases():
    _need_gpu()
    net = netkit.line(3, 300.0, 2)
    # all trips waiting at t = 0; nothing on the network
    dem = netkit.vehicles([-1] * 3, [0.0] * 3, [0.0] * 3, [[0, 1]] * 3, t_dep=[5, 5, 500])
    s = parity.gpu_sim(net, dem, P)
    o = oracle.Oracle(net, dem, P)
    s.step(4)
    o.run(4)
    assert s.read_state()["n_active"] == 0
    for _ in range(60):
        _, gd, gs, od, os_ = parity.step_pair(s, o)
        parity.compare_step(gd, gs, od, os_, dem.n)
    # a single vehicle that arrives: the network empties again
    dem1 = netkit.single(net, 0, 290.0, 15.0, [0])
    s1 = parity.gpu_sim(net, dem1, P)
    s1.step(1)
    st = s1.read_state()
    assert st["n_active"] == 0 and st["trip_status"][0] == 2 and st["t_arr"][0] == 1
    s1.step(3)   # stepping an empty network is fine
    s1.sync()


def test_invalid_inputs_are_rejected():
    _need_gpu()
    from paper_2405_12520_b300 import moss
    net = netkit.line(3, 300.0, 2)
    s = moss.Sim(P)
    s.load_network(net)
    bad = netkit.vehicles([-1], [0.0], [0.0], [[0, 2]])   # 0 -> 2 has no lane link (U-turn edge)
    with pytest.raises(moss.MossError) as e:
        s.add_vehicles(bad)
    assert e.value.code == moss.MS_ERR_ROUTE
    overlap = netkit.vehicles([0, 0], [100.0, 102.0], [0.0, 0.0], [[0, 1], [0, 1]])
    with pytest.raises(moss.MossError) as e:
        s.add_vehicles(overlap)
    assert e.value.code == moss.MS_ERR_ARG
    short = synth.grid_network(2, 2, 1, 30.0)
    short.lane_len[:] = 15.0   # shorter than v_max * dt
    s2 = moss.Sim(P)
    with pytest.raises(moss.MossError):
        s2.load_network(short)
    # an edge's lanes numbered from the left instead of the right: consistent left/right
    # links, but not the layout the lane-change search and the link plan index by
    flipped = netkit.line(3, 300.0, 2)
    l0 = int(flipped.edge_lane0[0])
    flipped.lane_left[l0], flipped.lane_right[l0] = -1, l0 + 1
    flipped.lane_left[l0 + 1], flipped.lane_right[l0 + 1] = l0, -1
    flipped.lane_index[l0], flipped.lane_index[l0 + 1] = 1, 0
    with pytest.raises(moss.MossError) as e:
        moss.Sim(P).load_network(flipped)
    assert e.value.code == moss.MS_ERR_ARG and "lane_index q" in str(e.value)
    wide = netkit.line(2, 300.0, 11)   # 11 lanes per edge: beyond the link plan's 10 fields
    with pytest.raises(moss.MossError) as e:
        moss.Sim(P).load_network(wide)
    assert e.value.code == moss.MS_ERR_CAPACITY and "10 lanes" in str(e.value)
    ten = netkit.line(2, 300.0, 10)    # the limit itself loads
    s3 = moss.Sim(P)
    s3.load_network(ten)
    s3.add_vehicles(netkit.vehicles([int(ten.edge_lane0[0]) + 9], [50.0], [10.0], [[0]]))
    s3.step(3)
    s3.sync()


def test_device_state_readout_into_torch():
    _need_gpu()
    import torch
    net, dem = synth.small_grid_workload(1)
    stream = torch.cuda.Stream()
    from paper_2405_12520_b300 import moss
    s = moss.Sim(P, stream=stream)
    s.load_network(net)
    s.add_vehicles(dem)
    s.step(100)
    x = torch.empty(dem.n, device="cuda")
    v = torch.empty_like(x)
    lane = torch.empty(dem.n, dtype=torch.int32, device="cuda")
    vid = torch.empty_like(lane)
    ri = torch.empty_like(lane)
    n = s.read_state_device(x, v, lane, vid, ri)
    st = s.read_state()
    torch.cuda.synchronize()
    assert n == st["n_active"]
    np.testing.assert_array_equal(x[:n].cpu().numpy(), st["x"])
    np.testing.assert_array_equal(vid[:n].cpu().numpy(), st["id"])
    np.testing.assert_array_equal(ri[:n].cpu().numpy(), st["route_idx"])


def test_async_state_export_overlaps_steps():
    """ms_read_state_async / ms_read_wait: the exported state equals the synchronous read of
    a twin simulation at the same step, with the export left in flight across one step (the
    overlapped pattern) and across several (the overwrite guard makes the steps wait)."""
    _need_gpu()
    import torch
    from paper_2405_12520_b300 import moss
    net, dem = synth.small_grid_workload(1)
    sims = []
    for _ in range(2):
        s = moss.Sim(P)
        s.load_network(net)
        s.add_vehicles(dem)
        sims.append(s)
    a, b = sims
    cap = dem.n
    bufs = [dict(x=torch.empty(cap, pin_memory=True), v=torch.empty(cap, pin_memory=True),
                 lane=torch.empty(cap, dtype=torch.int32, pin_memory=True),
                 vid=torch.empty(cap, dtype=torch.int32, pin_memory=True)) for _ in range(2)]

    def check(buf, n, t):
        st = b.read_state(trips=False)
        assert (n, t) == (st["n_active"], st["t"])
        np.testing.assert_array_equal(buf["x"][:n].numpy(), st["x"])
        np.testing.assert_array_equal(buf["v"][:n].numpy(), st["v"])
        np.testing.assert_array_equal(buf["lane"][:n].numpy(), st["lane"])
        np.testing.assert_array_equal(buf["vid"][:n].numpy(), st["id"])

    a.step(30)
    b.step(30)
    a.read_state_async(**bufs[0])
    for k in range(1, 40):                # export k-1 overlaps step k; step k+1 waits for it
        a.step(1)
        n, t = a.read_wait()
        check(bufs[(k - 1) % 2], n, t)
        b.step(1)
        a.read_state_async(**bufs[k % 2])
    n, t = a.read_wait()
    check(bufs[1], n, t)
    a.read_state_async(**bufs[0])         # two in flight: the second queues behind the first
    for k in range(1, 20):
        a.step(1)
        a.read_state_async(**bufs[k % 2])
        n, t = a.read_wait()              # the older one
        check(bufs[(k - 1) % 2], n, t)
        b.step(1)
    n, t = a.read_wait()
    check(bufs[1], n, t)
    a.read_state_async(**bufs[0])
    a.read_state_async(**bufs[1])
    with pytest.raises(moss.MossError) as e:
        a.read_state_async(**bufs[1])
    assert e.value.code == moss.MS_ERR_STATE
    check(bufs[0], *a.read_wait())
    check(bufs[1], *a.read_wait())
    a.read_state_async(**bufs[0])
    a.step(7)                             # steps past the exported buffer wait for the export
    n, t = a.read_wait()
    check(bufs[0], n, t)
    b.step(7)
    assert a.read_state(trips=False)["t"] == b.read_state(trips=False)["t"]
    with pytest.raises(moss.MossError) as e:
        a.read_wait()
    assert e.value.code == moss.MS_ERR_STATE
    small = {k: t[:5] for k, t in bufs[1].items()}
    a.read_state_async(**small)
    with pytest.raises(moss.MossError) as e:
        a.read_wait()
    assert e.value.code == moss.MS_ERR_CAPACITY
    np.testing.assert_array_equal(small["x"].numpy(), b.read_state(trips=False)["x"][:5])
    with pytest.raises(moss.MossError) as e:
        a.read_state_async(torch.empty(cap), None, None, None)
    assert e.value.code == moss.MS_ERR_ARG


def test_lane_speed_sums_on_long_lanes():
    """Per-lane window metrics of one step (sums of the snapshot's speeds, counts) against the
    oracle on lanes of 300, 150, 47, 31 and 1 vehicles: the parts of a lane past its first
    vehicle's warp are summed by that vehicle when at most 16 long (lane of 31) and by the
    whole warp when longer (300, 150, 47).  Counts are exact; a sum of n non-negative FP32
    speeds is within n * 2^-24 of the exact sum, relative."""
    _need_gpu()
    from paper_2405_12520_b300 import moss
    net = netkit.line(3, 2500.0, 3)
    l0 = [int(net.edge_lane0[0]) + q for q in range(3)]
    l2 = [int(net.edge_lane0[2]) + q for q in range(2)]
    rng = np.random.default_rng(11)
    lanes, xs, routes = [], [], []
    for l, cnt, route in ((l0[0], 300, [0, 1]), (l0[1], 150, [0, 1]), (l0[2], 47, [0, 1]),
                          (l2[0], 31, [2]), (l2[1], 1, [2])):
        lanes += [l] * cnt
        xs += list(10.0 + 8.0 * np.arange(cnt))
        routes += [route] * cnt
    vs = rng.uniform(0.0, 13.0, len(lanes))
    dem = netkit.vehicles(lanes, xs, vs, routes)
    sim = moss.Sim(P, debug=False, n_windows=1)
    sim.load_network(net)
    sim.add_vehicles(dem)
    st = sim.read_state()
    sim.step(1)
    sim.sync()
    gm = sim.read_metrics()
    orc = oracle.Oracle(net, dem, P, n_windows=1)
    orc.run(1)
    om = orc.metrics()
    np.testing.assert_array_equal(gm["vcnt"][0], om["vcnt"][0])
    cnt = om["vcnt"][0].astype(np.float64)
    assert sorted(cnt[cnt > 0].tolist()) == [1, 31, 47, 150, 300]
    gv, ov = gm["vsum"][0].astype(np.float64), om["vsum"][0]
    assert np.all(np.abs(gv - ov) <= cnt * 2.0 ** -24 * ov + 1e-6), np.abs(gv - ov).max()
    # the FP32 inputs summed exactly are the oracle's sums
    for l in (l0 + l2):
        sel = st["lane"] == l
        assert ov[l] == pytest.approx(float(np.sum(st["v"][sel].astype(np.float64))), rel=1e-12, abs=1e-9)


@pytest.mark.parametrize("kind,t0,mp", [("grid12x3", 12, False), ("delaunay", 5, False), ("grid12x3", 20, True)])
def test_single_steps_match_oracle_dynamic_lanes(kind, t0, mp):
    """About 30% of the lane links closed (R17) without disconnecting any route, set through
    the modification call on both sides (fixed-time and max-pressure signals)."""
    _need_gpu()
    net = _net(kind)
    prm = dict(P, signal_mode=1, mp_interval=10) if mp else P
    dem = synth.merge_demands(synth.place_vehicles(net, 5003 if kind == "grid12x3" else 2500, seed=61 + t0,
                                                   min_spacing=7.0, internal_frac=0.3),
                              synth.uniform_trips(net, 400, 40, seed=62 + t0))
    mask = netkit.closable_links(net, dem, np.random.default_rng(63 + t0), 0.3)
    lanes = np.array(list(mask), np.int32)
    masks = np.array([mask[int(l)] for l in lanes], np.uint32)
    n_closed = sum(int(np.diff(net.succ_off)[l]) - bin(int(m)).count("1") for l, m in zip(lanes, masks))
    assert n_closed > 0.2 * int(np.diff(net.succ_off)[lanes].sum())
    sim = parity.gpu_sim(net, dem, prm)
    st = sim.read_state()
    st["t"] = t0
    sim.write_state(st)
    orc = oracle.Oracle(net, dem, prm)
    sim.set_lane_links(lanes, masks)
    orc.set_lane_links(lanes, masks)
    rep = []
    for k in range(10):
        _, gd, gs, od, os_ = parity.step_pair(sim, orc)
        parity.compare_step(gd, gs, od, os_, dem.n, report=rep)
        if mp:
            np.testing.assert_array_equal(gs["ctrl_state"], os_["ctrl_state"])
    tot = {k: sum(r[k] for r in rep) for k in rep[0]}
    print(kind, mp, n_closed, tot)
    assert tot["compared"] > 0.9 * tot["active"]
    assert sim.read_metrics(lanes=False)["err"] == 0


def test_dynamic_lanes_successive_partial_calls_match_oracle():
    """Three calls that each touch about a tenth of the edges (close a set, close another,
    reopen the first), five single steps after each, under max-pressure signals with two of
    the calls on a decision step: the link plans of edges no call touched stay as they were,
    and the controllers retake the current step's decision over the links now open."""
    _need_gpu()
    net = _net("grid12x3")
    prm = dict(P, signal_mode=1, mp_interval=10)
    dem = synth.merge_demands(synth.place_vehicles(net, 5003, seed=91, min_spacing=7.0, internal_frac=0.3),
                              synth.uniform_trips(net, 400, 40, seed=92))
    rng = np.random.default_rng(93)
    mask = netkit.closable_links(net, dem, rng, 0.3)
    closing = [l for l, m in mask.items() if m != (1 << int(np.diff(net.succ_off)[l])) - 1]
    edges = np.unique(net.lane_edge[closing])
    pick = rng.permutation(edges)
    e_a, e_b = set(pick[: len(pick) // 8].tolist()), set(pick[len(pick) // 8: len(pick) // 4].tolist())
    set_a = [l for l in closing if int(net.lane_edge[l]) in e_a]
    set_b = [l for l in closing if int(net.lane_edge[l]) in e_b]
    assert len(set_a) > 10 and len(set_b) > 10
    full = {l: (1 << int(np.diff(net.succ_off)[l])) - 1 for l in set_a}
    calls = [(set_a, [mask[l] for l in set_a]), (set_b, [mask[l] for l in set_b]),
             (set_a, [full[l] for l in set_a])]
    sim = parity.gpu_sim(net, dem, prm)
    st = sim.read_state()
    st["t"] = 20
    sim.write_state(st)
    orc = oracle.Oracle(net, dem, prm)
    rep = []
    for lanes, masks in calls:
        lanes, masks = np.array(lanes, np.int32), np.array(masks, np.uint32)
        sim.set_lane_links(lanes, masks)
        orc.set_lane_links(lanes, masks)
        for k in range(5):
            _, gd, gs, od, os_ = parity.step_pair(sim, orc)
            parity.compare_step(gd, gs, od, os_, dem.n, report=rep)
            np.testing.assert_array_equal(gs["ctrl_state"], os_["ctrl_state"])
    tot = {k: sum(r[k] for r in rep) for k in rep[0]}
    print(len(set_a), len(set_b), tot)
    assert tot["compared"] > 0.9 * tot["active"]
    assert sim.read_metrics(lanes=False)["err"] == 0


def test_dynamic_lanes_reject_broken_routes_and_reopen_exactly():
    """Closing every link of the first edge toward the second breaks the routes of vehicles
    still to cross: MS_ERR_ROUTE and nothing changes.  Closing one lane's links forces its
    vehicles over; reopening every link gives the same steps as a simulation never
    modified."""
    _need_gpu()
    from paper_2405_12520_b300 import moss
    net = netkit.line(3, 300.0, 2)
    l0 = int(net.edge_lane0[0])
    dem = netkit.vehicles([l0, l0, l0 + 1], [60.0, 120.0, 90.0], [9.0, 8.0, 10.0], [[0, 1]] * 3)
    a = parity.gpu_sim(net, dem, P, debug=False)
    b = parity.gpu_sim(net, dem, P, debug=False)
    with pytest.raises(moss.MossError) as e:
        a.set_lane_links([l0, l0 + 1], [0, 0])
    assert e.value.code == moss.MS_ERR_ROUTE
    a.step(3)
    b.step(3)
    for k in ("id", "lane", "x", "v"):
        np.testing.assert_array_equal(a.read_state()[k], b.read_state()[k])
    a.set_lane_links([l0], [0])          # lane 0 no longer leads on: its vehicles change over
    a.step(40)
    sa = a.read_state()
    assert np.all(sa["lane"][sa["route_idx"] == 0] != l0)
    a.set_lane_links([l0], [0b11])       # reopened
    b.write_state(a.read_state())
    a.step(20)
    b.step(20)
    for k in ("id", "lane", "x", "v", "route_idx"):
        np.testing.assert_array_equal(a.read_state()[k], b.read_state()[k])
    with pytest.raises(moss.MossError) as e:
        a.set_lane_links([int(net.succ_lane[net.succ_off[l0]])], [1])   # an internal lane
    assert e.value.code == moss.MS_ERR_ARG


@pytest.mark.parametrize("t0", [0, 1])
def test_single_steps_match_oracle_on_long_lanes(t0):
    """Lanes of several hundred vehicles (3 km links, 3 lanes, random spacing down to 6 m):
    lane-change target searches over long segments, lanes spanning many warps in the
    apply's stayer ranks and the changers' bucket ranks, long remainders in the lane
    metrics; both step parities (left and right changes)."""
    _need_gpu()
    net = netkit.line(4, 3000.0, 3)
    rng = np.random.default_rng(70 + t0)
    lanes, xs, vs, routes = [], [], [], []
    # a dense slow lane, a sparse fast one and a medium one per edge: changes both ways
    mix = ((6.0, 9.0, 0.0, 4.0), (25.0, 45.0, 10.0, 14.0), (8.0, 12.0, 3.0, 7.0))
    for e, route in ((0, [0, 1, 2]), (1, [1, 2]), (5, [5, 4, 3])):
        for q, (g0, g1, v0_, v1_) in enumerate(mix):
            l = int(net.edge_lane0[e]) + q
            x = 8.0 + rng.uniform(0, 3)
            while x < 2990.0:
                lanes.append(l)
                xs.append(x)
                vs.append(rng.uniform(v0_, v1_))
                routes.append(route)
                x += rng.uniform(g0, g1)
    dem = netkit.vehicles(lanes, xs, vs, routes, v0=rng.uniform(11.0, 16.0, len(lanes)))
    cnt = np.bincount(np.asarray(lanes), minlength=net.n_lanes)
    assert cnt.max() > 250
    sim = parity.gpu_sim(net, dem, P, n_windows=1)
    st = sim.read_state()
    st["t"] = t0
    sim.write_state(st)
    orc = oracle.Oracle(net, dem, P, n_windows=1)
    rep = []
    for k in range(6):
        _, gd, gs, od, os_ = parity.step_pair(sim, orc)
        parity.compare_step(gd, gs, od, os_, dem.n, report=rep)
    tot = {k: sum(r[k] for r in rep) for k in rep[0]}
    print(t0, int(cnt.max()), tot)
    assert tot["compared"] > 0.95 * tot["active"] and tot["changes"] > 20
    assert sim.read_metrics(lanes=False)["err"] == 0


def test_standstill_queue_far_along_a_lane_resumes_exactly():
    """Bumper-to-bumper stopped vehicles 17 km along a lane (its next lane closed): their
    FP32 positions are multiples of 2e-3 m there, so exact gap-0 stops read back as gaps of
    about +-2e-3 m, which the state checks (ms_add_vehicles / ms_write_state and the debug
    order check) accept; resuming from the read state is bit-exact."""
    _need_gpu()
    net = netkit.line(3, 18000.0, 1)
    l0, l1 = int(net.edge_lane0[0]), int(net.edge_lane0[1])
    xs = np.float32(17000.1234) + np.float32(5.0) * np.arange(40, dtype=np.float32)
    xs[1::3] = np.nextafter(xs[1::3], np.float32(0))   # gaps of -1 ulp, as rounded clamps leave
    gap32 = np.diff(xs.astype(np.float64)) - P["veh_len"]
    assert gap32.min() < -1e-3                          # rounding beyond an absolute 1e-3
    dem = netkit.vehicles([l0] * 40, xs.astype(np.float64), [0.0] * 40, [[0, 1]] * 40)
    a = parity.gpu_sim(net, dem, P)                     # debug: device order / gap check
    b = parity.gpu_sim(net, dem, P)
    for s in (a, b):
        s.set_lane_limits([l1], closed=[1])
        s.step(20)
    st = a.read_state()
    a.write_state(st)
    a.step(20)
    b.step(20)
    sa, sb = a.read_state(), b.read_state()
    for k in ("id", "lane", "x", "v", "route_idx"):
        np.testing.assert_array_equal(sa[k], sb[k])
    assert a.read_metrics(lanes=False)["err"] == 0 and b.read_metrics(lanes=False)["err"] == 0


def test_whole_run_statistics_medium_grid():
    """A 20x20 grid (3 lanes, 300 m) with 40,000 vehicles on it and 20,000 trips departing
    over 600 s, free-running for 1200 steps on the GPU and in the FP64 oracle: completed
    trips, mean travel time and network mean speed per 5-minute window within 2%; per-lane
    5-minute mean speeds within 2% on average over lanes with >= 300 vehicle-steps."""
    _need_gpu()
    net = synth.grid_network(20, 20, 3, 300.0, 30, 3, "wave")
    dem = synth.merge_demands(synth.place_vehicles(net, 40_000, seed=21),
                              synth.gravity_trips(net, 20_000, t_span=600, seed=22))
    sim = parity.gpu_sim(net, dem, P, debug=False, n_windows=4)
    sim.step(1200)
    sim.sync()
    gm = sim.read_metrics()
    assert gm["err"] == 0
    orc = oracle.Oracle(net, dem, P, n_windows=4)
    orc.run(1200)
    om = orc.metrics()
    assert om["arrived"] > 10_000
    assert abs(gm["arrived"] - om["arrived"]) <= 0.02 * om["arrived"]
    assert abs(gm["sum_tt"] / gm["arrived"] - om["sum_tt"] / om["arrived"]) <= 0.02 * om["sum_tt"] / om["arrived"]
    gv, gc = gm["vsum"].astype(np.float64), gm["vcnt"].astype(np.float64)
    ov, oc = om["vsum"], om["vcnt"].astype(np.float64)
    net_g, net_o = gv.sum(1) / gc.sum(1), ov.sum(1) / oc.sum(1)
    assert np.all(np.abs(net_g - net_o) <= 0.02 * net_o), (net_g, net_o)
    m = (gc >= 300) & (oc >= 300)
    rel = np.abs(gv[m] / gc[m] - ov[m] / oc[m]) / np.maximum(ov[m] / oc[m], 1e-3)
    print("lanes compared", int(m.sum()), "mean rel", rel.mean(), "p90", np.quantile(rel, 0.9),
          "arrived", gm["arrived"], om["arrived"])
    assert m.sum() > 1000 and rel.mean() <= 0.02
