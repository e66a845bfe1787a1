"""Corner cases of the step, CUDA path against the FP64 oracle (through the C ABI).

Each case is one of the hand-built situations the oracle's pins fix in closed form (the
ballistic stop within a step and the gap clamp, a changer held at its lane end, the
12-lane cap of the look-ahead, the target lane's end at red, the mandatory change's tie,
departure timing and room behind the step's arrivals, the max-pressure tie between two
phases that are not green, the conflict guard, politeness with a target leader).  The GPU
steps from the same state as the oracle; every step is compared by parity.compare_step,
and the corner value itself is checked on the GPU's own output."""
import numpy as np
import pytest

import netkit
import oracle
import parity
from paper_2405_12520_b300 import synth

pytestmark = pytest.mark.gpu
P = synth.default_params()
MP = dict(P, signal_mode=1, mp_interval=10)


def _need_gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _pair(net, dem, params, t0=0, prep=None):
    sim = parity.gpu_sim(net, dem, params)
    orc = oracle.Oracle(net, dem, params)
    if t0:
        st = sim.read_state()
        st["t"] = t0
        sim.write_state(st)
    if prep:
        prep(sim)
        prep(orc)
    return sim, orc


def _steps(sim, orc, n_trips, k):
    out = []
    for _ in range(k):
        st0, gd, gs, od, os_ = parity.step_pair(sim, orc)
        parity.compare_step(gd, gs, od, os_, n_trips)
        out.append((st0, gd, gs, od, os_))
    return out


def _by_trip(gs, key, n):
    a = np.full(n, np.nan)
    a[gs["id"]] = gs[key]
    return a


def test_desired_speed_above_v_max_is_rejected():
    """The library accepts desired speeds in (0, v_max] only, so the v_max cap of the update
    (pinned on the oracle with a desired speed of 30 m/s) never binds on the device: a free
    vehicle approaches v0 <= v_max from below.  A trip above it is refused at the boundary."""
    _need_gpu()
    from paper_2405_12520_b300 import moss
    net = netkit.ring(200.0)
    dem = netkit.ring_demand(net, np.array([10.0]), np.array([0.0]), 30.0)
    sim = moss.Sim(P)
    sim.load_network(net)
    with pytest.raises(moss.MossError) as e:
        sim.add_vehicles(dem)
    assert e.value.code == moss.MS_ERR_ARG
    sim.destroy()


@pytest.mark.parametrize("v,gap,d_want,v_want", [(3.0, 3.0, 0.5, 0.0), (15.0, 4.0, 4.0, 4.0)])
def test_stop_within_the_step_and_gap_clamp(v, gap, d_want, v_want):
    _need_gpu()
    net = netkit.line(3, 300.0, 1)
    dem = netkit.vehicles([0, 0], [100.0, 100.0 + P["veh_len"] + gap], [v, 0.0], [[0, 1]] * 2)
    sim, orc = _pair(net, dem, P)
    st0, gd, gs, od, os_ = _steps(sim, orc, dem.n, 1)[0]
    assert gd["a_use"][0] == np.float32(P["a_min"])
    x = _by_trip(gs, "x", dem.n)
    vv = _by_trip(gs, "v", dem.n)
    assert abs(x[0] - 100.0 - d_want) <= 1e-5 and abs(vv[0] - v_want) <= 1e-5


def test_changer_held_at_its_lane_end():
    _need_gpu()
    net = netkit.line(4, 300.0, 2)
    l0, l1 = int(net.edge_lane0[0]), int(net.edge_lane0[1])
    il = [int(net.succ_lane[k]) for k in range(net.succ_off[l0], net.succ_off[l0 + 1])
          if net.succ_lane[net.succ_off[net.succ_lane[k]]] == l1][0]
    dem = netkit.vehicles([l0, l1], [295.0, 30.0 - float(net.lane_len[il])], [10.0, 5.0],
                          [[0, 1, 2], [1, 2]])
    sim, orc = _pair(net, dem, dict(P, x_lc_end=0.0))
    st0, gd, gs, od, os_ = _steps(sim, orc, dem.n, 1)[0]
    assert gd["lc_dir"][0] == 1
    lane = np.full(dem.n, -1)
    lane[gs["id"]] = gs["lane"]
    assert lane[0] == net.lane_left[l0]
    assert _by_trip(gs, "x", dem.n)[0] == 300.0 and abs(_by_trip(gs, "v", dem.n)[0] - 5.0) <= 1e-5


def test_lookahead_lane_cap():
    _need_gpu()
    net = netkit.line(20, 25.0, 1)
    l0 = int(net.edge_lane0[0])
    dem = netkit.vehicles([l0], [5.0], [10.0], [list(range(19))])
    sim, orc = _pair(net, dem, dict(P, d_look=1000.0))
    st0, gd, gs, od, os_ = _steps(sim, orc, dem.n, 1)[0]
    assert gd["lead_kind"][0] == 2 and od["lead_kind"][0] == 2
    assert abs(float(gd["s_own"][0]) - od["s_own"][0]) <= 1e-3


def test_target_lane_end_at_red():
    _need_gpu()
    net = synth.grid_network(3, 3, 2, 300.0, green=200, yellow=3, offset="zero")
    o0 = oracle.Oracle(net, netkit.vehicles([], [], [], []), P)
    case = None
    for e in range(net.n_edges):
        l = int(net.edge_lane0[e])
        if net.edge_to[e] != 4 or net.edge_nlanes[e] != 2 or o0.signal_state(l, 0) != 2:
            continue
        both = set(net.succ_edge[net.succ_off[l]:net.succ_off[l + 1]]) & set(
            net.succ_edge[net.succ_off[l + 1]:net.succ_off[l + 2]])
        if both:
            case = (e, l, int(sorted(both)[0]))
            break
    e, l, ex = case
    xc = float(net.lane_len[l]) - 30.0
    dem = netkit.vehicles([l, l], [xc, xc + P["veh_len"] + 3.0], [0.0, 0.0], [[e, ex]] * 2)
    sim, orc = _pair(net, dem, P)
    st0, gd, gs, od, os_ = _steps(sim, orc, dem.n, 1)[0]
    want = P["idm_a"] * P["idm_s0"] ** 2 * (1 / 9.0 - 1 / 900.0)
    assert gd["lc_cand"][0] == 1 and abs(float(gd["incentive"][0]) - want) <= 1e-4


@pytest.mark.parametrize("t0,want_cand,want_dir", [(0, 0, 0), (1, 1, -1)])
def test_mandatory_change_tie(t0, want_cand, want_dir):
    _need_gpu()
    net = netkit.line(3, 300.0, 3)
    mid = int(net.edge_lane0[0]) + 1
    dem = netkit.vehicles([mid], [150.0], [10.0], [[0, 1]])
    sim, orc = _pair(net, dem, P, t0=t0, prep=lambda o: o.set_lane_links([mid], [0]))
    st0, gd, gs, od, os_ = _steps(sim, orc, dem.n, 1)[0]
    assert gd["lc_cand"][0] == want_cand and gd["lc_dir"][0] == want_dir


def test_departure_at_its_time_and_room_behind_arrivals():
    _need_gpu()
    # a lone trip due at t = 5 on an empty road enters at the step whose clock is 5
    net = netkit.line(3, 300.0, 1)
    dem = netkit.vehicles([-1], [0.0], [0.0], [[0, 1]], t_dep=[5])
    sim, orc = _pair(net, dem, P)
    recs = _steps(sim, orc, dem.n, 8)
    assert [int(r[1]["inserted"][0]) for r in recs] == [0, 0, 0, 0, 0, 1, 0, 0]
    # an arrival landing 11 m into the departure lane leaves no room (rear 6 m < L + s0)
    net = netkit.line(4, 300.0, 1)
    l0, l1 = int(net.edge_lane0[0]), int(net.edge_lane0[1])
    il = int(net.succ_lane[net.succ_off[l0]])
    v = 12.0
    a = P["idm_a"] * (1 - (v / float(np.float32(13.9))) ** 4)
    x = float(net.lane_len[il]) - (0.5 * (2 * v + a) - 11.0)
    dem = netkit.vehicles([il, -1], [x, 0.0], [v, 0.0], [[0, 1, 2], [1, 2]], t_dep=[0, 0])
    sim, orc = _pair(net, dem, P)
    recs = _steps(sim, orc, dem.n, 3)
    assert [int(r[1]["inserted"][1]) for r in recs] == [0, 0, 1]


def test_max_pressure_tie_between_two_other_phases():
    _need_gpu()
    net = synth.delaunay_network(60, seed=3)
    lanes_of = lambda c: np.nonzero((net.lane_ctrl == c) & (net.lane_edge >= 0))[0]
    ctrl = next(c for c in range(net.n_ctrl) if net.ctrl_nphase[c] >= 3 and
                {0, 1, 2} <= set(net.lane_group[lanes_of(c)].tolist()))
    ls = lanes_of(ctrl)
    la, lb = int(ls[net.lane_group[ls] == 1][0]), int(ls[net.lane_group[ls] == 2][0])
    na, nb = (int(net.succ_off[l + 1] - net.succ_off[l]) for l in (la, lb))
    lanes, xs, routes = [], [], []
    for l, k in ((la, nb), (lb, na)):
        for q in range(k):
            lanes.append(l)
            xs.append(float(net.lane_len[l]) - 10.0 - 8.0 * q)
            routes.append([int(net.lane_edge[l]), int(net.succ_edge[net.succ_off[l]])])
    dem = netkit.vehicles(lanes, xs, [0.0] * len(lanes), routes)
    sim, orc = _pair(net, dem, MP)
    recs = _steps(sim, orc, dem.n, 5)
    # after the step at t = 0 phase 0 is yellow with phase 1 pending, the lower of the tie
    assert recs[0][2]["ctrl_state"][ctrl].tolist()[:2] == [0, 1]


def test_conflict_guard_and_politeness_with_a_target_leader():
    _need_gpu()
    net = netkit.line(3, 300.0, 2)
    L = P["veh_len"]
    stopped = 100.0 + L + 3.0
    cases = [([0, 0, 1], [100.0, stopped, 100.0 - L - 2.5], [12.0, 0.0, 2.0], 0),
             ([0, 0, 1], [100.0, stopped, 100.0 - L - 3.5], [12.0, 0.0, 2.0], 1),
             ([0, 0, 1, 1], [100.0, 100.0 + L + 2.5, 100.0 + L + 3.0, 100.0 - L - 3.0], [0.0] * 4, None)]
    for lanes, xs, vs, want in cases:
        dem = netkit.vehicles(lanes, xs, vs, [[0, 1]] * len(lanes))
        sim, orc = _pair(net, dem, P)
        st0, gd, gs, od, os_ = _steps(sim, orc, dem.n, 1)[0]
        assert gd["lc_cand"][0] == 1
        if want is not None:
            assert gd["lc_dir"][0] == want
        else:
            assert abs(float(gd["incentive"][0]) - od["incentive"][0]) <= 1e-4


def test_level_vehicle_in_the_target_lane_is_the_follower():
    _need_gpu()
    net = netkit.line(3, 300.0, 2)
    dem = netkit.vehicles([0, 0, 1, 1], [100.0, 108.0, 100.0, 130.0], [5.0, 0.0, 5.0, 5.0], [[0, 1]] * 4)
    sim, orc = _pair(net, dem, P)
    st0, gd, gs, od, os_ = _steps(sim, orc, dem.n, 1)[0]
    assert gd["lc_cand"][0] == 1 and gd["tau_foll"][0] == 2 and gd["tau_lead"][0] == 3
    assert gd["lc_dir"][0] == 0


def test_departures_by_time_and_onto_the_first_linked_lane():
    _need_gpu()
    # one departure lane, departure times 8, 6, 4, 2, 0: entries in time order
    net = netkit.line(3, 300.0, 1)
    dem = netkit.vehicles([-1] * 5, [0.0] * 5, [0.0] * 5, [[0, 1]] * 5, t_dep=[8, 6, 4, 2, 0])
    sim, orc = _pair(net, dem, P)
    order = []
    for r in _steps(sim, orc, dem.n, 60):
        order += np.nonzero(r[1]["inserted"])[0].tolist()
    assert order == [4, 3, 2, 1, 0]
    # 3-lane approaches whose lane 0 serves only the right turn: every trip enters the
    # lowest lane of its first edge linked to its second edge
    net = synth.grid_network(3, 3, 3, 300.0, green=30, yellow=3)
    trips = []
    for e in range(net.n_edges):
        l0 = int(net.edge_lane0[e])
        links = lambda q: net.succ_edge[net.succ_off[l0 + q]:net.succ_off[l0 + q + 1]]
        for f in sorted({int(f) for q in range(int(net.edge_nlanes[e])) for f in links(q)}):
            trips.append(([e, f], min(l0 + q for q in range(int(net.edge_nlanes[e])) if f in links(q))))
    n = len(trips)
    dem = netkit.vehicles([-1] * n, [0.0] * n, [0.0] * n, [r for r, _ in trips], t_dep=[2 * k for k in range(n)])
    sim, orc = _pair(net, dem, P)
    entry = {}
    for r in _steps(sim, orc, dem.n, 2 * n + 20):
        gs = r[2]
        lane = np.full(n, -1)
        lane[gs["id"]] = gs["lane"]
        for i in np.nonzero(r[1]["inserted"])[0]:
            entry[int(i)] = int(lane[i])
    assert len(entry) == n and all(entry[k] == w for k, (_, w) in enumerate(trips))


def test_fan_out_fallback_with_closed_links():
    _need_gpu()
    net = synth.grid_network(3, 3, 3, 300.0, green=30, yellow=3)
    e = [k for k in range(net.n_edges) if net.edge_from[k] == 3 and net.edge_to[k] == 4][0]
    ex = [k for k in range(net.n_edges) if net.edge_from[k] == 4 and net.edge_to[k] == 5][0]
    mid = int(net.edge_lane0[e]) + 1
    tg = [int(net.succ_lane[net.succ_off[net.succ_lane[k]]]) for k in range(net.succ_off[mid], net.succ_off[mid + 1])]
    keep = tg.index(int(net.edge_lane0[ex]) + 2)
    l_ex0 = int(net.edge_lane0[ex])
    serves = lambda l, f: f in net.succ_edge[net.succ_off[l]:net.succ_off[l + 1]]
    after = [int(f) for f in net.succ_edge[net.succ_off[l_ex0]:net.succ_off[l_ex0 + 1]]
             if not serves(l_ex0 + 2, int(f))][0]
    dem = netkit.vehicles([mid], [290.0], [8.0], [[e, ex, after]])
    sim, orc = _pair(net, dem, P, prep=lambda o: o.set_lane_links([mid], [1 << keep]))
    _steps(sim, orc, dem.n, 80)


def test_target_lane_end_at_yellow_with_a_follower():
    _need_gpu()
    net = synth.grid_network(3, 3, 2, 300.0, green=200, yellow=3, offset="zero")
    o0 = oracle.Oracle(net, netkit.vehicles([], [], [], []), P)
    case = None
    for e in range(net.n_edges):
        l = int(net.edge_lane0[e])
        if net.edge_to[e] != 4 or net.edge_nlanes[e] != 2 or o0.signal_state(l, 200) != 1:
            continue
        both = set(net.succ_edge[net.succ_off[l]:net.succ_off[l + 1]]) & set(
            net.succ_edge[net.succ_off[l + 1]:net.succ_off[l + 2]])
        if both:
            case = (e, l, int(sorted(both)[0]))
            break
    e, l, ex = case
    L = P["veh_len"]
    xc = float(net.lane_len[l]) - 30.0
    dem = netkit.vehicles([l, l, l + 1], [xc, xc + L + 3.0, xc - L - 3.0], [0.0] * 3, [[e, ex]] * 3)
    sim, orc = _pair(net, dem, P, t0=200)
    st0, gd, gs, od, os_ = _steps(sim, orc, dem.n, 1)[0]
    assert gd["lc_cand"][0] == 1 and gd["tau_foll"][0] == 2
    assert abs(float(gd["incentive"][0]) - od["incentive"][0]) <= 1e-4


@pytest.mark.parametrize("limited_lane, trail_lane", [(0, 0), (1, 1)])
def test_followers_under_lane_limits(limited_lane, trail_lane):
    _need_gpu()
    net = netkit.line(3, 300.0, 2)
    L = P["veh_len"]
    dem = netkit.vehicles([0, 0, trail_lane], [100.0, 100.0 + L + 10.0, 100.0 - L - 10.0], [8.0, 0.0, 8.0],
                          [[0, 1]] * 3)
    sim, orc = _pair(net, dem, P, prep=lambda o: o.set_lane_limits([limited_lane], vmax=[8.0]))
    st0, gd, gs, od, os_ = _steps(sim, orc, dem.n, 1)[0]
    assert gd["lc_cand"][0] == 1
    assert abs(float(gd["incentive"][0]) - od["incentive"][0]) <= 1e-4


@pytest.mark.parametrize("t0", [0, 1])
def test_discretionary_target_must_serve_the_route(t0):
    _need_gpu()
    net = synth.grid_network(3, 3, 3, 300.0, green=30, yellow=3)
    e = [k for k in range(net.n_edges) if net.edge_from[k] == 3 and net.edge_to[k] == 4][0]
    ex = [k for k in range(net.n_edges) if net.edge_from[k] == 4 and net.edge_to[k] == 5][0]
    l0 = int(net.edge_lane0[e])
    dem = netkit.vehicles([l0 + 1, l0 + 1], [100.0, 108.0], [5.0, 0.0], [[e, ex]] * 2)
    sim, orc = _pair(net, dem, P, t0=t0)
    st0, gd, gs, od, os_ = _steps(sim, orc, dem.n, 1)[0]
    assert gd["lc_cand"][0] == 0 and gd["lc_dir"][0] == 0


def test_max_pressure_decisions_inside_a_yellow_are_refused():
    """The oracle pins max pressure deciding every 2 s inside a 3 s yellow; the library takes
    decision intervals longer than every controller's yellow only, so on the device a
    decision never meets a pending switch, and such a network is refused."""
    _need_gpu()
    from paper_2405_12520_b300 import moss
    net, dem = synth.small_grid_workload(2)
    sim = moss.Sim(dict(MP, mp_interval=2))
    with pytest.raises(moss.MossError) as e:
        sim.load_network(net)
    assert e.value.code == moss.MS_ERR_ARG
    sim.destroy()


def test_rewinding_a_run_resumes_it_exactly():
    _need_gpu()
    net, dem = synth.small_grid_workload(3)
    sim = parity.gpu_sim(net, dem, P, debug=False)
    sim.step(200)
    s200 = sim.read_state()
    sim.step(200)
    sim.sync()
    end = sim.read_state()
    sim.write_state(s200)
    sim.step(200)
    sim.sync()
    again = sim.read_state()
    for k in ("id", "lane", "x", "v", "route_idx", "trip_status", "t_arr"):
        assert np.array_equal(end[k], again[k]), k
    assert end["t"] == again["t"]
