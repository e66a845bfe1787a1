"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
published RNG vectors, closed forms of the IDM (Treiber 2000) and of MOBIL special cases
(Kesting 2007), the fixed-time signal table, brute-force neighbour search, and invariants
of whole runs (gap >= 0, no crossing on red, conservation, determinism, resume)."""
import math
import os

import numpy as np
import pytest
from scipy.optimize import brentq

from paper_2405_12520_b300 import synth
import netkit

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
P = synth.default_params()


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            rows.append(line.split())
    return rows


# ---------------------------------------------------------------------------------------
# counter-based RNG
# ---------------------------------------------------------------------------------------

def test_splitmix64_published_vector(oracle_lib):
    """SplitMix64 (Steele, Lea & Flood 2014) seeded with 0: the first outputs are the
    published reference values.  The oracle's function is the output step applied to the
    state, so the k-th output is f(k * gamma)."""
    gamma = 0x9E3779B97F4A7C15
    for k, (hexval,) in enumerate(_golden("splitmix64_seed0.txt")):
        assert oracle_lib.splitmix64((k * gamma) % 2 ** 64) == int(hexval, 16)


# ---------------------------------------------------------------------------------------
# IDM closed forms
# ---------------------------------------------------------------------------------------

def _equilibrium_speed(gap, v0, p=P):
    """Treiber's homogeneous steady state: s_e(v) = (s0 + vT) / sqrt(1 - (v/v0)^4)."""
    f = lambda v: (p["idm_s0"] + v * p["idm_T"]) / math.sqrt(1.0 - (v / v0) ** 4) - gap
    return brentq(f, 0.0, v0 * (1 - 1e-12), xtol=1e-15, rtol=1e-15)


@pytest.mark.parametrize("n_veh", [16, 20, 40])
def test_idm_ring_equilibrium_is_fixed_point(oracle_lib, n_veh):
    net = netkit.ring(200.0)
    _, _, total = netkit.ring_path(net)
    spacing = total / n_veh
    gap = spacing - P["veh_len"]
    v0 = 13.9
    ve = _equilibrium_speed(gap, v0)
    u = 0.5 + spacing * np.arange(n_veh)   # ring is 460 m: these fronts are exact in float32
    dem = netkit.ring_demand(net, u, np.full(n_veh, ve), v0)
    o = oracle_lib.Oracle(net, dem, P)
    seq, starts, _ = netkit.ring_path(net)
    lane_start = {l: s for l, s in zip(seq, starts)}

    def ring_pos(st):
        return np.array([lane_start[l] + x for l, x in zip(st["lane"], st["x"])])
    moved = 0.0
    for k in range(50):
        before = ring_pos(o.state())
        err, d = o.step(debug=True)
        assert err == 0
        # speeds enter as float32 (ve rounded by ~5e-7), hence 1e-6 rather than 0
        assert np.all(np.abs(d["a_own"]) < 1e-6), np.abs(d["a_own"]).max()
        assert np.all(d["lead_kind"] == 1)
        np.testing.assert_allclose(d["s_own"], gap, atol=1e-4)
        st = o.state()
        adv = np.mod(ring_pos(st) - before, total)
        np.testing.assert_allclose(adv, ve * P["dt"], atol=1e-6)
        np.testing.assert_allclose(st["v"], ve, atol=1e-6)
        moved += adv.mean()
    assert moved > 0


def test_free_road_accelerates_to_v0(oracle_lib):
    net = netkit.ring(200.0)
    v0 = 13.9
    dem = netkit.ring_demand(net, np.array([10.0]), np.array([0.0]), v0)
    o = oracle_lib.Oracle(net, dem, P)
    seq, starts, total = netkit.ring_path(net)
    lane_start = {l: s for l, s in zip(seq, starts)}
    vs, us = [0.0], [10.0]
    for k in range(300):
        _, d = o.step(debug=True)
        assert d["lead_kind"][0] == 0   # ring is longer than the look-ahead horizon
        st = o.state()
        vs.append(st["v"][0])
        us.append(lane_start[st["lane"][0]] + st["x"][0])
    vs = np.array(vs)
    # first step from rest: a = a_max exactly, so v = a_max dt and d = a_max dt^2 / 2
    assert vs[1] == pytest.approx(P["idm_a"] * P["dt"], abs=1e-12)
    assert np.mod(us[1] - us[0], total) == pytest.approx(0.5 * P["idm_a"], abs=1e-12)
    v0f = float(np.float32(v0))   # desired speeds are float32 inputs
    assert np.all(np.diff(vs) >= 0) and np.all(np.diff(vs[:30]) > 0) and np.all(vs <= v0f)
    assert vs[-1] == pytest.approx(v0f, abs=1e-9)
    # ballistic update: distance of each step is the mean of the two speeds times dt
    adv = np.mod(np.diff(us), total)
    np.testing.assert_allclose(adv, 0.5 * (vs[1:] + vs[:-1]) * P["dt"], atol=1e-9)


def test_motion_stop_within_the_step_and_gap_clamp(oracle_lib):
    """The ballistic update's two corner cases on a one-lane road behind a stopped leader,
    where IDM asks for far more than a_min = -9 m/s^2 and the clamp to a_min holds:
    at 3 m/s and a 3 m gap the vehicle stops within the step after v^2 / (2 |a_min|) =
    0.5 m; at 15 m/s and a 4 m gap the ballistic distance 0.5 (15 + 6) = 10.5 m is cut to
    the gap and the speed to gap / dt = 4 m/s."""
    net = netkit.line(3, 300.0, 1)
    L, am = P["veh_len"], P["a_min"]
    for v, gap, d_want, v_want in ((3.0, 3.0, 9.0 / 18.0, 0.0), (15.0, 4.0, 4.0, 4.0)):
        dem = netkit.vehicles([0, 0], [100.0, 100.0 + L + gap], [v, 0.0], [[0, 1]] * 2)
        o = oracle_lib.Oracle(net, dem, P)
        x0 = o.state()["x"][0]
        _, d = o.step(debug=True)
        assert d["lead_id"][0] == 1 and d["a_use"][0] == am
        st = o.state()
        assert st["x"][0] - x0 == pytest.approx(d_want, abs=1e-12)
        assert st["v"][0] == pytest.approx(v_want, abs=1e-12)


def test_speed_is_capped_at_v_max(oracle_lib):
    """A lone vehicle whose desired speed (30 m/s) is above v_max (20 m/s) on a free ring
    accelerates to v_max and stays there: the update caps v' at v_max."""
    net = netkit.ring(200.0)
    dem = netkit.ring_demand(net, np.array([10.0]), np.array([0.0]), 30.0)
    o = oracle_lib.Oracle(net, dem, P)
    vs = []
    for _ in range(60):
        o.step()
        vs.append(o.state()["v"][0])
    assert max(vs) == P["v_max"] and vs[-1] == P["v_max"] and vs[9] < P["v_max"]


def test_changer_stops_at_its_lane_end(oracle_lib):
    """A discretionary change 5 m before the lane end (the end zone set to 0): the own path
    continues to a slower leader 30 m ahead on the next edge, the target lane is free, so
    the vehicle changes; it moves at most to the end of its lane in that step, so at 10 m/s
    its distance is cut to 5 m and its speed to 5 m/s."""
    net = netkit.line(4, 300.0, 2)
    l0, l1 = int(net.edge_lane0[0]), int(net.edge_lane0[1])
    il = [int(net.succ_lane[k]) for k in range(net.succ_off[l0], net.succ_off[l0 + 1])
          if net.succ_lane[net.succ_off[net.succ_lane[k]]] == l1][0]
    x_lead = 30.0 - float(net.lane_len[il])     # own gap (5 + len(il) + x_lead) - L = 30 m
    dem = netkit.vehicles([l0, l1], [300.0 - 5.0, x_lead], [10.0, 5.0], [[0, 1, 2], [1, 2]])
    o = oracle_lib.Oracle(net, dem, dict(P, x_lc_end=0.0))
    _, d = o.step(debug=True)
    assert d["lead_id"][0] == 1 and d["s_own"][0] == pytest.approx(30.0, abs=1e-9)
    assert d["lc_dir"][0] == +1 and d["a_use"][0] > 0.0
    st = o.state()
    assert st["lane"][0] == net.lane_left[l0]
    assert st["x"][0] == 300.0 and st["v"][0] == pytest.approx(5.0, abs=1e-12)


def test_lookahead_ends_at_the_twelfth_lane(oracle_lib):
    """On a road of 25 m links (21 m junction lanes) with a 1 km look-ahead, an empty path
    ends the look-ahead after 12 lanes, the own lane included: the end of the 12th lane is a
    stopped obstacle at the summed lengths of the path."""
    net = netkit.line(20, 25.0, 1)
    l0 = int(net.edge_lane0[0])
    dem = netkit.vehicles([l0], [5.0], [10.0], [list(range(19))])
    o = oracle_lib.Oracle(net, dem, dict(P, d_look=1000.0))
    _, d = o.step(debug=True)
    path, cur = [l0], l0
    while len(path) < 12:
        k = [k for k in range(net.succ_off[cur], net.succ_off[cur + 1])][0]
        cur = int(net.succ_lane[k])
        path.append(cur)
    want = (25.0 - 5.0) + float(np.sum(net.lane_len[path[1:]].astype(np.float64)))
    assert d["lead_kind"][0] == 2 and d["s_own"][0] == pytest.approx(want, abs=1e-9)


def test_motion_and_the_conflict_guard_scale_with_dt(oracle_lib):
    """With a time step of 0.5 s: from rest on a free road the first step gives v' = a_max dt
    and d = a_max dt^2 / 2; at 15 m/s 4 m behind a stopped leader (IDM clamped at a_min)
    the ballistic distance 0.5 (15 + 10.5) dt = 6.375 m is cut to the gap and the speed to
    gap / dt = 8 m/s; and the conflict guard of a follower at 4 m/s is
    v_F dt + a_max dt^2 / 2 = 2.25 m (a changer at 14 m/s keeps the follower's IDM desired gap
    at s0, so only the guard decides between 2.2 and 2.4 m)."""
    dt, am, L = 0.5, P["idm_a"], P["veh_len"]
    Pd = dict(P, dt=dt)
    net = netkit.ring(200.0)
    dem = netkit.ring_demand(net, np.array([10.0]), np.array([0.0]), 13.9)
    o = oracle_lib.Oracle(net, dem, Pd)
    x0 = o.state()["x"][0]
    o.step()
    st = o.state()
    assert st["v"][0] == pytest.approx(am * dt, abs=1e-12)
    assert st["x"][0] - x0 == pytest.approx(0.5 * am * dt * dt, abs=1e-12)
    line = netkit.line(3, 300.0, 1)
    dem = netkit.vehicles([0, 0], [100.0, 100.0 + L + 4.0], [15.0, 0.0], [[0, 1]] * 2)
    o = oracle_lib.Oracle(line, dem, Pd)
    _, d = o.step(debug=True)
    assert d["a_use"][0] == P["a_min"]
    st = o.state()
    assert st["x"][0] == pytest.approx(104.0, abs=1e-12) and st["v"][0] == pytest.approx(4.0 / dt, abs=1e-12)
    stopped = 100.0 + L + 3.0
    for g, allowed in ((2.2, False), (2.4, True)):
        assert am * (1 - (4.0 / 13.9) ** 4 - (P["idm_s0"] / g) ** 2) > -P["mobil_bsafe"]
        d = _two_lane_case([0, 0, 1], [100.0, stopped, 100.0 - L - g], [14.0, 0.0, 4.0], dt=dt)
        assert d["lc_cand"][0] == 1 and d["tau_foll"][0] == 2
        assert d["lc_dir"][0] == (+1 if allowed else 0), g


def test_target_lane_end_at_yellow_takes_the_stopping_distance(oracle_lib):
    """At the first second of yellow a changer at 10 m/s, 15 m before the line (it can stop:
    v^2 / (2 b) = 11.1 m), with both lanes ending at that line: the target lane's end blocks
    it as its own lane's does, so the prospective and the present acceleration are the same
    IDM value before a stopped obstacle 15 m ahead and the incentive is exactly 0."""
    net = synth.grid_network(3, 3, 2, 300.0, green=200, yellow=3, offset="zero")
    o0 = oracle_lib.Oracle(net, netkit.vehicles([], [], [], []), P)
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
    dem = netkit.vehicles([l], [float(net.lane_len[l]) - 15.0], [10.0], [[e, ex]])
    o = oracle_lib.Oracle(net, dem, dict(P, x_lc_end=0.0))
    st = o.state()
    o.set_state(st["status"], st["lane"], st["x"], st["v"], st["rp"], 200)
    _, d = o.step(debug=True)
    assert 15.0 >= 10.0 ** 2 / (2 * P["idm_b"])
    assert d["lead_kind"][0] == 2 and d["s_own"][0] == pytest.approx(15.0, abs=1e-9)
    assert d["lc_cand"][0] == 1 and d["tau_lead"][0] == -1
    assert d["incentive"][0] == 0.0


def test_stop_at_long_red_reaches_standstill_gap(oracle_lib):
    net = synth.grid_network(3, 3, 1, 300.0, green=200, yellow=3, offset="zero")
    o0 = oracle_lib.Oracle(net, netkit.vehicles([], [], [], []), P)
    # an approach lane into the centre node (4) that is red for t in [0, 203)
    lanes = [l for l in range(net.n_edge_lanes)
             if net.edge_to[net.lane_edge[l]] == 4 and o0.signal_state(l, 0) == 2]
    l = lanes[0]
    e = net.lane_edge[l]
    nxt = [net.succ_edge[k] for k in range(net.succ_off[l], net.succ_off[l + 1])][0]
    dem = netkit.vehicles([l], [100.0], [12.0], [[e, nxt]])
    o = oracle_lib.Oracle(net, dem, P)
    L = net.lane_len[l]
    for t in range(200):
        o.step()
        st = o.state()
        assert st["lane"][0] == l and st["x"][0] <= L   # never crosses the red stop line
    st = o.state()
    # standing still short of the line: with a discrete step the stop can end a little
    # inside s0, where IDM then gives a < 0 and the vehicle stays put
    assert st["v"][0] == 0.0
    assert 0.0 < (L - st["x"][0]) <= P["idm_s0"] + 1e-9
    for t in range(200, 260):
        o.step()
    assert o.state()["lane"][0] != l or o.state()["status"][0] == 2   # left on green


def test_signal_table_closed_form(oracle_lib):
    net = synth.grid_network(3, 3, 1, 300.0, green=30, yellow=3, offset="zero")
    o = oracle_lib.Oracle(net, netkit.vehicles([], [], [], []), P)
    c = net.ctrl_node.tolist().index(4)
    lanes = np.nonzero(net.lane_ctrl == c)[0]
    g0 = [l for l in lanes if net.lane_group[l] == 0][0]
    g1 = [l for l in lanes if net.lane_group[l] == 1][0]
    want0 = ["G"] * 30 + ["Y"] * 3 + ["R"] * 33
    want1 = ["R"] * 33 + ["G"] * 30 + ["Y"] * 3
    code = {0: "G", 1: "Y", 2: "R"}
    for t in range(132):
        assert code[o.signal_state(g0, t)] == want0[t % 66]
        assert code[o.signal_state(g1, t)] == want1[t % 66]
    # uncontrolled lanes (corner nodes have fewer than 3 approaches) are always green
    free = np.nonzero(net.lane_ctrl[:net.n_edge_lanes] < 0)[0][0]
    assert all(o.signal_state(free, t) == 0 for t in range(70))


def test_signal_offsets_shift_the_table(oracle_lib):
    """An offset of o seconds advances a controller's plan by o: with the green-wave
    offsets, a lane's state at t is the state the same lane has at t + o in the same grid
    with every offset 0 (whose table the closed-form pin above fixes)."""
    wave = synth.grid_network(4, 4, 1, 300.0, green=30, yellow=3, offset="wave")
    zero = synth.grid_network(4, 4, 1, 300.0, green=30, yellow=3, offset="zero")
    np.testing.assert_array_equal(wave.lane_ctrl, zero.lane_ctrl)
    np.testing.assert_array_equal(wave.lane_group, zero.lane_group)
    ow = oracle_lib.Oracle(wave, netkit.vehicles([], [], [], []), P)
    oz = oracle_lib.Oracle(zero, netkit.vehicles([], [], [], []), P)
    shifted = 0
    for c in range(wave.n_ctrl):
        n = wave.ctrl_node[c]
        off = ((n % 4) + (n // 4)) * 22 % (wave.ctrl_nphase[c] * 33)
        assert wave.ctrl_offset[c] == off and zero.ctrl_offset[c] == 0
        shifted += off != 0
        for l in np.nonzero(wave.lane_ctrl == c)[0]:
            for t in range(140):
                assert ow.signal_state(int(l), t) == oz.signal_state(int(l), t + int(off)), (c, l, t)
    assert shifted > 0


def test_yellow_stop_rule(oracle_lib):
    """At the start of yellow a vehicle stops iff its distance to the stop line is at
    least v^2 / (2 b)."""
    net = synth.grid_network(3, 3, 1, 300.0, green=30, yellow=3, offset="zero")
    o0 = oracle_lib.Oracle(net, netkit.vehicles([], [], [], []), P)
    lanes = [l for l in range(net.n_edge_lanes)
             if net.edge_to[net.lane_edge[l]] == 4 and o0.signal_state(l, 30) == 1]
    v = 15.0
    stop_d = v * v / (2 * P["idm_b"])   # 25 m
    routes, xs, ls = [], [], []
    for l, dist in zip(lanes[:2], [stop_d + 5.0, stop_d - 5.0]):
        e = net.lane_edge[l]
        nxt = net.succ_edge[net.succ_off[l]]
        routes.append([e, nxt])
        xs.append(net.lane_len[l] - dist)
        ls.append(l)
    dem = netkit.vehicles(ls, xs, [v, v], routes)
    o = oracle_lib.Oracle(net, dem, P)
    st = o.state()
    o.set_state(st["status"], st["lane"], st["x"], st["v"], st["rp"], 30)
    _, d = o.step(debug=True)
    assert d["lead_kind"][0] == 2 and d["s_own"][0] == pytest.approx(stop_d + 5.0)
    assert d["lead_kind"][1] != 2


# ---------------------------------------------------------------------------------------
# MOBIL special cases
# ---------------------------------------------------------------------------------------

def _two_lane_case(lanes, xs, vs, v0=13.9, t=0, **par):
    net = netkit.line(3, 300.0, 2)
    routes = [[0, 1]] * len(lanes)
    dem = netkit.vehicles(lanes, xs, vs, routes, v0=v0)
    import oracle
    o = oracle.Oracle(net, dem, dict(P, **par))
    if t:
        st = o.state()
        o.set_state(st["status"], st["lane"], st["x"], st["v"], st["rp"], t)
    err, d = o.step(debug=True)
    assert err == 0
    return d


def test_mobil_incentive_is_free_gain_with_empty_target(oracle_lib):
    v, v0 = 10.0, 13.9
    se = (P["idm_s0"] + v * P["idm_T"]) / math.sqrt(1 - (v / v0) ** 4)   # Treiber s_e(v)
    d = _two_lane_case([0, 0], [100.0, 100.0 + P["veh_len"] + se], [v, v])
    # inputs are float32 (positions, v0): equilibrium and free gain hold to ~1e-7
    v0f = float(np.float32(v0))
    assert d["a_own"][0] == pytest.approx(0.0, abs=1e-6)   # car-following equilibrium
    assert d["lc_cand"][0] == 1
    assert d["tau_lead"][0] == -1 and d["tau_foll"][0] == -1 and d["old_foll"][0] == -1
    assert d["incentive"][0] == pytest.approx(P["idm_a"] * (1 - (v / v0f) ** 4), abs=1e-6)
    assert d["lc_dir"][0] == +1
    # a changer moves with the lower of its current and prospective accelerations
    assert d["a_use"][0] == d["a_own"][0]


def test_mobil_identical_lanes_no_change(oracle_lib):
    v, v0 = 10.0, 13.9
    se = (P["idm_s0"] + v * P["idm_T"]) / math.sqrt(1 - (v / v0) ** 4)
    xl = 100.0 + P["veh_len"] + se
    d = _two_lane_case([0, 0, 1], [100.0, xl, xl], [v, v, v])
    assert d["lc_cand"][0] == 1 and d["tau_lead"][0] == 2
    assert d["incentive"][0] == 0.0
    assert d["lc_dir"][0] == 0


def test_mobil_direction_alternates_with_step_parity(oracle_lib):
    v, v0 = 10.0, 13.9
    se = (P["idm_s0"] + v * P["idm_T"]) / math.sqrt(1 - (v / v0) ** 4)
    # vehicle on the left lane (1) behind a leader: on even steps only left moves exist
    d = _two_lane_case([1, 1], [100.0, 100.0 + 5 + se], [v, v], t=0)
    assert d["lc_cand"][0] == 0
    d = _two_lane_case([1, 1], [100.0, 100.0 + 5 + se], [v, v], t=1)
    assert d["lc_cand"][0] == 1 and d["lc_dir"][0] == -1


def test_mobil_safety_criteria(oracle_lib):
    stopped_leader = 100.0 + P["veh_len"] + 3.0
    # new follower 10 m behind at 8.5 m/s: guard 9.5 m passes, a~_n < -b_safe blocks
    d = _two_lane_case([0, 0, 1], [100.0, stopped_leader, 85.0], [5.0, 0.0, 8.5])
    assert d["lc_cand"][0] == 1 and d["tau_foll"][0] == 2 and d["lc_dir"][0] == 0
    # same with a stopped follower: a~_n = a_max (1 - (s0/10)^2) = 1.92 > -b_safe: change
    d = _two_lane_case([0, 0, 1], [100.0, stopped_leader, 85.0], [5.0, 0.0, 0.0])
    assert d["lc_dir"][0] == +1
    # conflict guard: follower 9.5 m behind at 9 m/s needs 9 + a_max/2 = 10 m
    d = _two_lane_case([0, 0, 1], [100.0, stopped_leader, 85.5], [5.0, 0.0, 9.0])
    assert d["lc_cand"][0] == 1 and d["lc_dir"][0] == 0
    # the guard alone: a changer at 12 m/s closes so fast on a follower at 2 m/s that the
    # follower's IDM desired gap is s0 (v T + v dv / (2 sqrt(a b)) = 3 - 3.33 < 0), so at a
    # gap g its deceleration a_max (1 - (2/13.9)^4 - (s0/g)^2) is mild for g >= 2.25 m; the
    # guard v_F dt + a_max dt^2 / 2 = 3 m still rejects g = 2.5 m and admits g = 3.5 m
    am, s0, L = P["idm_a"], P["idm_s0"], P["veh_len"]
    for g, allowed in ((2.5, False), (3.5, True)):
        assert am * (1 - (2.0 / 13.9) ** 4 - (s0 / g) ** 2) > -P["mobil_bsafe"]
        d = _two_lane_case([0, 0, 1], [100.0, stopped_leader, 100.0 - L - g], [12.0, 0.0, 2.0])
        assert d["lc_cand"][0] == 1 and d["tau_foll"][0] == 2
        assert d["lc_dir"][0] == (+1 if allowed else 0), g


def test_mobil_zones_and_gate(oracle_lib):
    stopped = P["veh_len"] + 3.0
    # too close to the lane start (x < x_lc_min = 25 m), and just past it
    d = _two_lane_case([0, 0], [20.0, 20.0 + stopped], [5.0, 0.0])
    assert d["lc_cand"][0] == 0
    d = _two_lane_case([0, 0], [26.0, 26.0 + stopped], [5.0, 0.0])
    assert d["lc_cand"][0] == 1
    # too close to the lane end for a discretionary change (len - x < x_lc_end = 20 m), and
    # just outside that zone
    d = _two_lane_case([0, 0], [285.0, 285.0 + 2], [5.0, 0.0])
    assert d["lc_cand"][0] == 0
    d = _two_lane_case([0, 0], [279.0, 279.0 + stopped], [5.0, 0.0])
    assert d["lc_cand"][0] == 1
    # p_lc = 0: never considered
    d = _two_lane_case([0, 0], [100.0, 100.0 + stopped], [5.0, 0.0], p_lc=0.0)
    assert d["lc_cand"][0] == 0


def test_random_gate_is_a_fresh_draw_per_trip_and_step(oracle_lib):
    """With p_lc = 0.3, 400 vehicles that pass every other candidate test (each 59 m apart on
    one long 2-lane road, at equilibrium behind its leader, the left lane free) become
    candidates with probability 0.3 each, drawn afresh at every step: at each of two even
    steps the share is 0.3 within 4 binomial standard deviations, and the share that pass
    at both is 0.09 within the same margin (independent draws)."""
    n, p = 400, 0.3
    v, v0 = 10.0, 13.9
    se = (P["idm_s0"] + v * P["idm_T"]) / math.sqrt(1 - (v / v0) ** 4)
    net = netkit.line(2, 24000.0, 2)
    xs, vs = [], []
    for q in range(n):
        base = 60.0 + 59.0 * q
        xs += [base, base + P["veh_len"] + se]
        vs += [v, v]
    dem = netkit.vehicles([0] * (2 * n), xs, vs, [[0]] * (2 * n), v0=v0)
    import oracle
    picks = []
    for t0 in (0, 2):
        o = oracle.Oracle(net, dem, dict(P, p_lc=p, x_lc_end=0.0))
        st = o.state()
        o.set_state(st["status"], st["lane"], st["x"], st["v"], st["rp"], t0)
        _, d = o.step(debug=True)
        picks.append(d["lc_cand"][0::2] == 1)
    for pk in picks:
        assert abs(pk.mean() - p) <= 4 * math.sqrt(p * (1 - p) / n)
    both = (picks[0] & picks[1]).mean()
    assert abs(both - p * p) <= 4 * math.sqrt(p * p * (1 - p * p) / n)


JITTER_SALT = 0x9E3779B97F4A7C15


def _trip_u(oracle_lib, seed, trip):
    """The trip's 24-bit uniform of the threshold-jitter variant, from the published
    SplitMix64 (pinned above)."""
    return (oracle_lib.splitmix64((seed ^ JITTER_SALT ^ trip) % 2 ** 64) >> 40) / 2.0 ** 24


def test_mobil_threshold_jitter_per_trip(oracle_lib):
    """Free-gain case (incentive a_max(1 - (v/v0)^4), closed form): with the jitter variant
    the change happens exactly when the incentive beats the trip's threshold
    th + J(2u - 1), for seeds whose draws fall on both sides."""
    v, v0, J = 10.0, 13.9, 2.0
    se = (P["idm_s0"] + v * P["idm_T"]) / math.sqrt(1 - (v / v0) ** 4)
    gain = P["idm_a"] * (1 - (v / float(np.float32(v0))) ** 4)
    seen = set()
    for seed in range(1, 41):
        th = P["mobil_th"] + J * (2 * _trip_u(oracle_lib, seed, 0) - 1)
        if abs(gain - th) < 1e-3:
            continue
        d = _two_lane_case([0, 0], [100.0, 100.0 + P["veh_len"] + se], [v, v], seed=seed, mobil_th_jitter=J)
        assert d["incentive"][0] == pytest.approx(gain, abs=1e-6)
        want = +1 if gain > th else 0
        assert d["lc_dir"][0] == want, (seed, th)
        seen.add(want)
    assert seen == {0, 1}
    # jitter 0: the plain threshold, whatever the seed
    d = _two_lane_case([0, 0], [100.0, 100.0 + P["veh_len"] + se], [v, v], seed=7, mobil_th=gain + 0.01)
    assert d["lc_dir"][0] == 0


def test_mobil_threshold_jitter_is_uniform_over_trips(oracle_lib):
    """Many independent free-gain pairs (one per edge of a long road): the share of
    followers that change matches P(th + J(2u - 1) < gain) = (gain - th + J) / (2J) for a
    uniform u, within 4 standard deviations; without jitter all of them change."""
    import oracle
    n_nodes, v, v0, J = 400, 10.0, 13.9, 2.0
    net = netkit.line(n_nodes, 300.0, 2)
    se = (P["idm_s0"] + v * P["idm_T"]) / math.sqrt(1 - (v / v0) ** 4)
    lanes, xs, routes = [], [], []
    for e in range(n_nodes - 1):   # edges 0 .. n-2 run k -> k+1
        l0 = int(net.edge_lane0[e])
        lanes += [l0, l0]
        xs += [100.0, 100.0 + P["veh_len"] + se]
        r = [e, e + 1] if e + 1 < n_nodes - 1 else [e]
        routes += [r, r]
    dem = netkit.vehicles(lanes, xs, [v] * len(lanes), routes, v0=v0)
    gain = P["idm_a"] * (1 - (v / float(np.float32(v0))) ** 4)
    share = {}
    for jit in (0.0, J):
        o = oracle.Oracle(net, dem, dict(P, mobil_th_jitter=jit, seed=11))
        err, d = o.step(debug=True)
        assert err == 0
        foll = np.arange(0, dem.n, 2)
        assert np.allclose(d["incentive"][foll], gain, atol=1e-6)
        share[jit] = float(np.mean(d["lc_dir"][foll] == 1))
    assert share[0.0] == 1.0
    p = (gain - P["mobil_th"] + J) / (2 * J)
    sd = math.sqrt(p * (1 - p) / (n_nodes - 1))
    assert abs(share[J] - p) <= 4 * sd, (share[J], p)


def test_mandatory_change_toward_connecting_lane(oracle_lib):
    """A 3-lane approach whose lane 0 serves only the right turn: a vehicle on lane 0
    heading straight must move left, with no incentive test."""
    net = synth.grid_network(3, 3, 3, 300.0, green=30, yellow=3)
    # approach into node 4 from the west: edge 3 -> 4
    e = [k for k in range(net.n_edges) if net.edge_from[k] == 3 and net.edge_to[k] == 4][0]
    ex = [k for k in range(net.n_edges) if net.edge_from[k] == 4 and net.edge_to[k] == 5][0]
    l0 = net.edge_lane0[e]
    serves = lambda l: ex in net.succ_edge[net.succ_off[l]:net.succ_off[l + 1]]
    assert not serves(l0) and serves(l0 + 1)
    # free road, no reason to change except the route
    dem = netkit.vehicles([l0], [150.0], [13.9], [[e, ex]])   # lane end 150 m ahead
    import oracle
    o = oracle.Oracle(net, dem, P)
    _, d = o.step(debug=True)
    assert d["lead_kind"][0] == 2   # non-connecting lane end is an obstacle
    assert d["lc_dir"][0] == +1 and d["lc_cand"][0] == 1
    o2 = oracle.Oracle(net, dem, dict(P, p_lc=0.0))
    _, d2 = o2.step(debug=True)
    assert d2["lc_dir"][0] == +1    # mandatory changes bypass the random gate


def test_fan_out_falls_back_to_the_first_open_link(oracle_lib):
    """The middle lane of a 3-lane approach links to all three lanes of the straight exit;
    with two of those links closed, the only open one leads to the exit's left lane, which
    does not serve the right turn the route takes after it.  No link of the lane reaches
    a lane serving the edge after next, so the vehicle takes the first open link to its next
    edge (and changes lanes there): it crosses onto the exit's left lane."""
    net = synth.grid_network(3, 3, 3, 300.0, green=30, yellow=3)
    e = [k for k in range(net.n_edges) if net.edge_from[k] == 3 and net.edge_to[k] == 4][0]
    ex = [k for k in range(net.n_edges) if net.edge_from[k] == 4 and net.edge_to[k] == 5][0]
    mid = int(net.edge_lane0[e]) + 1
    links = [(int(net.succ_lane[k]), int(net.succ_lane[net.succ_off[net.succ_lane[k]]]))
             for k in range(net.succ_off[mid], net.succ_off[mid + 1])]
    left_exit = int(net.edge_lane0[ex]) + 2
    keep = [j for j, (_, tgt) in enumerate(links) if tgt == left_exit]
    assert len(keep) == 1 and len(links) == 3
    # the edge after the exit: one its left lane does not serve, but another exit lane does
    serves = lambda l, f: f in net.succ_edge[net.succ_off[l]:net.succ_off[l + 1]]
    after = [int(f) for f in net.succ_edge[net.succ_off[int(net.edge_lane0[ex])]:
                                            net.succ_off[int(net.edge_lane0[ex]) + 1]]
             if not serves(left_exit, int(f))][0]
    dem = netkit.vehicles([mid], [290.0], [8.0], [[e, ex, after]])
    o = oracle_lib.Oracle(net, dem, P)
    o.set_lane_links([mid], [1 << keep[0]])
    seen = []
    for _ in range(120):
        o.step()
        st = o.state()
        if st["status"][0] == 1 and (not seen or seen[-1] != int(st["lane"][0])):
            seen.append(int(st["lane"][0]))
    assert links[keep[0]][0] in seen and left_exit in seen
    assert seen.index(left_exit) == seen.index(links[keep[0]][0]) + 1


def test_mandatory_change_tie_goes_to_the_lower_lane(oracle_lib):
    """Three lanes, the middle lane's links to the next edge closed: the two lanes that still
    connect are equally near, and the lower index (the right lane) is the one to reach, so
    the change waits for a step that allows moves to the right."""
    net = netkit.line(3, 300.0, 3)
    l0 = int(net.edge_lane0[0])
    mid = l0 + 1
    dem = netkit.vehicles([mid], [150.0], [10.0], [[0, 1]])
    import oracle
    for t0, want_cand, want_dir in ((0, 0, 0), (1, 1, -1)):
        o = oracle.Oracle(net, dem, P)
        o.set_lane_links([mid], [0])
        st = o.state()
        o.set_state(st["status"], st["lane"], st["x"], st["v"], st["rp"], t0)
        _, d = o.step(debug=True)
        assert d["lc_cand"][0] == want_cand and d["lc_dir"][0] == want_dir, t0
    assert net.lane_right[mid] == l0


def test_target_lane_end_at_red_is_an_obstacle(oracle_lib):
    """A stopped vehicle 30 m before a red stop line, 3 m behind a stopped leader, with an
    empty target lane that also ends at the red line: the prospective acceleration is IDM
    against a stopped obstacle at the target lane's end (v = 0: a_max (1 - (s0/30)^2)), not
    the free road, so the incentive is a_max s0^2 (1/9 - 1/900)."""
    net = synth.grid_network(3, 3, 2, 300.0, green=200, yellow=3, offset="zero")
    o0 = oracle_lib.Oracle(net, netkit.vehicles([], [], [], []), P)
    L, s0, am = P["veh_len"], P["idm_s0"], P["idm_a"]
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
    assert case is not None
    e, l, ex = case
    assert o0.signal_state(l + 1, 0) == 2 and net.lane_left[l] == l + 1
    xc = float(net.lane_len[l]) - 30.0
    dem = netkit.vehicles([l, l], [xc, xc + L + 3.0], [0.0, 0.0], [[e, ex]] * 2)
    o = oracle_lib.Oracle(net, dem, P)
    _, d = o.step(debug=True)
    assert d["lc_cand"][0] == 1 and d["tau_lead"][0] == -1 and d["lead_id"][0] == 1
    assert d["incentive"][0] == pytest.approx(am * s0 ** 2 * (1 / 9.0 - 1 / 900.0), abs=1e-9)


def test_target_lane_end_at_yellow_and_the_followers_old_gap(oracle_lib):
    """At the first second of yellow, everybody stopped (v = 0: IDM is a_max (1 - (s0/s)^2)
    and every vehicle can stop): the changer 30 m before the stop line, 3 m behind its
    leader, a follower 3 m behind it in the empty target lane.  The target lane's end is a
    stopped obstacle for both: the changer's prospective gap is 30 m, the follower's present
    gap is its distance to the line, 30 + L + 3 m."""
    net = synth.grid_network(3, 3, 2, 300.0, green=200, yellow=3, offset="zero")
    o0 = oracle_lib.Oracle(net, netkit.vehicles([], [], [], []), P)
    L, s0, am, pol = P["veh_len"], P["idm_s0"], P["idm_a"], P["mobil_p"]
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
    assert case is not None
    e, l, ex = case
    xc = float(net.lane_len[l]) - 30.0
    dem = netkit.vehicles([l, l, l + 1], [xc, xc + L + 3.0, xc - L - 3.0], [0.0] * 3, [[e, ex]] * 3)
    o = oracle_lib.Oracle(net, dem, P)
    st = o.state()
    o.set_state(st["status"], st["lane"], st["x"], st["v"], st["rp"], 200)
    _, d = o.step(debug=True)
    idm0 = lambda gap: am * (1 - (s0 / gap) ** 2)
    want = idm0(30.0) - idm0(3.0) + pol * (idm0(3.0) - idm0(30.0 + L + 3.0))
    assert d["lc_cand"][0] == 1 and d["tau_lead"][0] == -1 and d["tau_foll"][0] == 2
    assert d["incentive"][0] == pytest.approx(want, abs=1e-9)


def test_idm_below_one_metre_of_gap(oracle_lib):
    """Two vehicles standing 0.9 m apart: the follower's IDM acceleration is the formula's
    a_max (1 - (s0 / 0.9)^2) = -7.88 m/s^2 (above a_min, so not clamped); the 0.01 m floor
    of the gap does not reach it."""
    d = _two_lane_case([0, 0], [100.0, 100.0 + P["veh_len"] + 0.9], [0.0, 0.0])
    g = float(np.float32(100.0 + P["veh_len"] + 0.9)) - 100.0 - P["veh_len"]
    want = P["idm_a"] * (1 - (P["idm_s0"] / g) ** 2)
    assert P["a_min"] < want < -7.0
    assert d["a_own"][0] == pytest.approx(want, abs=1e-9)


# ---------------------------------------------------------------------------------------
# neighbour search vs brute force
# ---------------------------------------------------------------------------------------

def _brute_neighbours(net, lane, x, active):
    n = lane.shape[0]
    out = np.full((n, 6), -1, np.int64)
    for c in np.nonzero(active)[0]:
        same = np.nonzero(active & (lane == lane[c]))[0]
        ahead = same[x[same] > x[c]]
        behind = same[x[same] < x[c]]
        if ahead.size:
            out[c, 0] = ahead[np.argmin(x[ahead])]
        if behind.size:
            out[c, 1] = behind[np.argmax(x[behind])]
        for q, tau in enumerate((net.lane_left[lane[c]], net.lane_right[lane[c]])):
            if tau < 0:
                continue
            oth = np.nonzero(active & (lane == tau))[0]
            a = oth[x[oth] > x[c]]
            b = oth[x[oth] <= x[c]]
            if a.size:
                out[c, 2 + 2 * q] = a[np.argmin(x[a])]
            if b.size:
                out[c, 3 + 2 * q] = b[np.argmax(x[b])]
    return out


@pytest.mark.parametrize("kind,seed", [("grid", 1), ("grid", 2), ("delaunay", 3)])
def test_neighbours_match_brute_force(oracle_lib, kind, seed):
    if kind == "grid":
        net = synth.grid_network(4, 4, 3, 200.0)
    else:
        net = synth.delaunay_network(40, box=2000.0, seed=seed)
    dem = synth.place_vehicles(net, 60, seed=seed, min_spacing=5.5, internal_frac=0.3)
    o = oracle_lib.Oracle(net, dem, P)
    got = o.neighbors()
    st = o.state()
    want = _brute_neighbours(net, st["lane"], st["x"], st["status"] == 1)
    np.testing.assert_array_equal(got, want)


def _r11_next(net, l, en, en2):
    """R11: among edge lane l's links toward edge en (CSR order), the first whose target lane
    links to en2 (any if en2 < 0), else the first; -1 if none."""
    first = -1
    for k in range(net.succ_off[l], net.succ_off[l + 1]):
        if net.succ_edge[k] != en:
            continue
        il = int(net.succ_lane[k])
        if first < 0:
            first = il
        if en2 < 0:
            return il
        tg = int(net.succ_lane[net.succ_off[il]])
        if any(net.succ_edge[q] == en2 for q in range(net.succ_off[tg], net.succ_off[tg + 1])):
            return il
    return first


def _brute_leaders(net, dem, st, d_look, L):
    """Own-path leader of every active vehicle by brute force, as path coordinates over ALL
    vehicles: the lanes the route passes through (R11 choices) from the vehicle's lane, each
    with the path coordinate of its start, as long as a lane starts less than d_look ahead
    of the vehicle's front; the leader is the vehicle with the smallest path coordinate ahead
    of the front, gap = its coordinate - L - x.  No vehicle: a stopped obstacle if the path
    ended at a lane without a link toward the next route edge, else free.  Then R3's merge
    projection: on an internal lane whose target has other feeders, on each of them the
    vehicle nearest the merge point among those farther from it... (d_j < d or d_j == d with
    a lower id), gap d - d_j - L, wins when smaller.  Networks without signals."""
    act = np.nonzero(st["status"] == 1)[0]
    lane, x, rp = st["lane"], st["x"], st["rp"]
    ln = np.asarray(net.lane_len, np.float64)
    edge = np.asarray(net.lane_edge)
    kind = np.zeros(dem.n, np.int64)
    lead = np.full(dem.n, -1, np.int64)
    gap = np.zeros(dem.n)
    for c in act:
        route = dem.route_edges[dem.route_off[c]:dem.route_off[c + 1]]
        at = lambda k: int(route[k]) if 0 <= k < route.shape[0] else -1
        path = [(int(lane[c]), 0.0)]
        cur, ri, start, blocked = int(lane[c]), int(rp[c]), 0.0, False
        while start + ln[cur] - x[c] < d_look:
            if edge[cur] >= 0:
                en = at(ri + 1)
                if en < 0:
                    break                          # destination edge: open end
                nxt = _r11_next(net, cur, en, at(ri + 2))
                if nxt < 0:
                    blocked = True
                    break
            else:
                nxt = int(net.succ_lane[net.succ_off[cur]])
                ri += 1
            start += ln[cur]
            path.append((nxt, start))
            cur = nxt
        assert len(path) <= 11                     # the 12-lane cap is not reached here
        best, bu = -1, np.inf
        for (pl, s0) in path:
            on = act[(lane[act] == pl) & (act != c)]
            u = s0 + x[on]
            if pl == lane[c]:
                keep = x[on] > x[c]
                on, u = on[keep], u[keep]
            if on.size and u.min() < bu:
                bu, best = float(u.min()), int(on[np.argmin(u)])
        if best >= 0:
            kind[c], lead[c], gap[c] = 1, best, bu - L - x[c]
        elif blocked:
            kind[c], gap[c] = 2, (path[-1][1] + ln[path[-1][0]]) - x[c]
        l = int(lane[c])
        if edge[l] < 0:                            # R3
            tgt = int(net.succ_lane[net.succ_off[l]])
            feeders = [f for f in range(net.n_lanes)
                       if edge[f] < 0 and int(net.succ_lane[net.succ_off[f]]) == tgt]
            if len(feeders) > 1:
                dc = ln[l] - x[c]
                for f in feeders:
                    if f == l:
                        continue
                    on = act[lane[act] == f]
                    dj = ln[f] - x[on]
                    ok = (dj < dc) | ((dj == dc) & (on < c))
                    if not ok.any():
                        continue
                    j = on[ok][np.argmax(dj[ok])]
                    g = (dc - (ln[f] - x[j])) - L
                    if kind[c] == 0 or g < gap[c]:
                        kind[c], lead[c], gap[c] = 1, j, g
    return kind, lead, gap


@pytest.mark.parametrize("kind,seed,t0", [("grid", 4, 0), ("grid", 5, 1), ("delaunay", 6, 0), ("delaunay", 7, 1)])
def test_step_leaders_and_target_neighbours_match_brute_force(oracle_lib, kind, seed, t0):
    """or_step's own sensing (R2 look-ahead across lane ends, R3 merges) and its lane-change
    target neighbours, read from its debug record, against brute force over all vehicles on
    random states with many vehicles near lane ends and on junction lanes."""
    if kind == "grid":
        net = synth.grid_network(4, 4, 2, 120.0, 30, 3, "zero")
    else:
        net = synth.delaunay_network(40, box=2000.0, seed=seed)
    net.lane_ctrl = np.full(net.n_lanes, -1, np.int32)     # no signals: obstacles are missing links
    dem = synth.place_vehicles(net, 90 if kind == "grid" else 220, seed=seed, min_spacing=5.5,
                               internal_frac=0.4)
    o = oracle_lib.Oracle(net, dem, P)
    st = o.state()
    o.set_state(st["status"], st["lane"], st["x"], st["v"], st["rp"], t0, st["t_arr"])
    _, d = o.step(debug=True)
    k_b, lead_b, gap_b = _brute_leaders(net, dem, st, P["d_look"], P["veh_len"])
    act = np.nonzero(st["status"] == 1)[0]
    np.testing.assert_array_equal(d["lead_kind"][act], k_b[act])
    np.testing.assert_array_equal(d["lead_id"][act], lead_b[act])
    has = act[k_b[act] != 0]
    np.testing.assert_allclose(d["s_own"][has], gap_b[has], rtol=0, atol=1e-9)
    assert (k_b[act] == 1).sum() > 20 and (k_b[act] == 2).sum() + (k_b[act] == 0).sum() > 3
    ahead_next = sum(1 for c in act if k_b[c] == 1 and st["lane"][lead_b[c]] != st["lane"][c])
    assert ahead_next > 10                         # leaders found across lane ends
    # lane-change target neighbours of the candidates (lane l+1 on even steps, l-1 on odd)
    nb = _brute_neighbours(net, st["lane"], st["x"], st["status"] == 1)
    side = 0 if t0 % 2 == 0 else 1
    cand = act[d["lc_cand"][act] == 1]
    assert cand.size > 5
    np.testing.assert_array_equal(d["tau_lead"][cand], nb[cand, 2 + 2 * side])
    np.testing.assert_array_equal(d["tau_foll"][cand], nb[cand, 3 + 2 * side])
    of = act[d["old_foll"][act] >= 0]
    np.testing.assert_array_equal(d["old_foll"][of], nb[of, 1])


# ---------------------------------------------------------------------------------------
# max-pressure signals (R13)
# ---------------------------------------------------------------------------------------

MP = dict(P, signal_mode=1, mp_interval=10)


def _center_lanes(net, ctrl):
    """Approach edge lanes of controller ctrl, by phase group."""
    ls = np.nonzero((net.lane_ctrl == ctrl) & (net.lane_edge >= 0))[0]
    return {int(g): ls[net.lane_group[ls] == g] for g in np.unique(net.lane_group[ls])}


def test_max_pressure_switches_to_the_loaded_phase(oracle_lib):
    """3x3 grid, only the centre's approach from the west (phase 1) holds a queue: at the
    decision step t = 0 phase 0 turns yellow for the controller's 3 s, then phase 1 is
    green until the next decision."""
    import oracle
    net = synth.grid_network(3, 3, 2, 200.0, 30, 3, "zero")
    ctrl = int(np.nonzero(net.ctrl_node == 4)[0][0])
    groups = _center_lanes(net, ctrl)
    e_in = int(np.nonzero((net.edge_from == 3) & (net.edge_to == 4))[0][0])
    e_out = int(np.nonzero((net.edge_from == 4) & (net.edge_to == 5))[0][0])
    l0 = int(net.edge_lane0[e_in])
    assert set(groups[1].tolist()) >= {l0, l0 + 1}
    lanes, xs = [], []
    for k in range(4):
        lanes += [l0, l0 + 1]
        xs += [190.0 - 8.0 * k] * 2
    dem = netkit.vehicles(lanes, xs, [0.0] * len(lanes), [[e_in, e_out]] * len(lanes))
    o = oracle.Oracle(net, dem, MP)
    seen = []
    for t in range(8):
        cs = o.ctrl_state()[ctrl].tolist()
        seen.append((o.signal_state(int(groups[0][0]), t), o.signal_state(int(groups[1][0]), t), cs))
        err, _ = o.step()
        assert err == 0
    Y, G, R = 1, 0, 2
    assert [x[:2] for x in seen[:3]] == [(Y, R)] * 3
    assert [x[:2] for x in seen[3:8]] == [(R, G)] * 5
    assert seen[0][2] == [0, 1, 3] and seen[3][2] == [1, -1, 3]


def test_max_pressure_holds_the_green_phase_on_ties(oracle_lib):
    """No vehicle anywhere near the controllers: every pressure is 0 and every controller
    keeps its green phase through many decisions (a fixed-time plan would have cycled),
    phase 0 from the start and phase 1 once set to it."""
    import oracle
    net = synth.grid_network(3, 3, 2, 200.0, 30, 3, "zero")
    e01 = int(np.nonzero((net.edge_from == 0) & (net.edge_to == 1))[0][0])
    dem = netkit.vehicles([-1], [0.0], [0.0], [[e01]], t_dep=[10 ** 6])   # departs far in the future
    o = oracle.Oracle(net, dem, MP)
    for t in range(60):
        assert (o.ctrl_state() == np.array([0, -1, 0])).all()
        o.step()
    # a tie keeps the phase that is green, not the lowest: every controller set to phase 1
    # holds it through six more decisions
    o.set_ctrl_state(np.tile([1, -1, 0], (net.n_ctrl, 1)))
    for t in range(60):
        o.step()
        assert (o.ctrl_state() == np.array([1, -1, 0])).all()


def test_max_pressure_tie_between_two_other_phases_goes_to_the_lower(oracle_lib):
    """A controller of a Delaunay city with three or more phases, phase 0 green with empty
    approaches, and phases 1 and 2 loaded to the same pressure (one approach lane each, the
    counts inverse to the lanes' link counts, nothing downstream): the decision at t = 0
    turns to phase 1, the lower index of the tie."""
    import oracle
    net = synth.delaunay_network(60, seed=3)
    ctrl = next(c for c in range(net.n_ctrl) if net.ctrl_nphase[c] >= 3 and
                {0, 1, 2} <= set(_center_lanes(net, c)))
    groups = _center_lanes(net, ctrl)
    la, lb = int(groups[1][0]), int(groups[2][0])
    na, nb = (int(net.succ_off[l + 1] - net.succ_off[l]) for l in (la, lb))
    lanes, xs, routes = [], [], []
    for l, k in ((la, nb), (lb, na)):                 # pressures na * nb on both phases
        assert 8.0 * k + 10.0 < net.lane_len[l]
        for q in range(k):
            lanes.append(l)
            xs.append(float(net.lane_len[l]) - 10.0 - 8.0 * q)
            routes.append([int(net.lane_edge[l]), int(net.succ_edge[net.succ_off[l]])])
    dem = netkit.vehicles(lanes, xs, [0.0] * len(lanes), routes)
    o = oracle.Oracle(net, dem, MP)
    # the controllers' state at t = 0 includes that step's decision: phase 1 pending
    assert o.ctrl_state()[ctrl].tolist()[:2] == [0, 1]


def test_max_pressure_steps_advance_the_controllers_themselves(oracle_lib):
    """Reading the controllers' state is an observation, not a step: a max-pressure run that
    reads them before every step and one that never does end in the same state, bit for
    bit, after 800 steps with switches in them."""
    import oracle
    net, dem = synth.small_grid_workload(2)
    a = oracle.Oracle(net, dem, MP)
    b = oracle.Oracle(net, dem, MP)
    seen = set()
    for _ in range(800):
        seen.add(tuple(a.ctrl_state()[:, 0].tolist()))
        a.step()
        b.step()
    assert len(seen) > 3
    sa, sb = a.state(), b.state()
    for k in ("status", "lane", "x", "v", "rp", "t_arr"):
        assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(a.ctrl_state(), b.ctrl_state())


def _mp_brute(net, counts, cs_prev, t, interval):
    """R13 restated with numpy over the network arrays, from the previous step's state."""
    cs = cs_prev.copy()
    for c in range(net.n_ctrl):
        if cs[c, 1] >= 0 and t >= cs[c, 2]:
            cs[c, 0], cs[c, 1] = cs[c, 1], -1
    if t % interval:
        return cs
    ls = np.nonzero((net.lane_ctrl >= 0) & (net.lane_edge >= 0))[0]
    pres = np.zeros((net.n_ctrl, int(net.ctrl_nphase.max())), np.int64)
    for l in ls:
        il = net.succ_lane[net.succ_off[l]:net.succ_off[l + 1]]
        tg = net.succ_lane[net.succ_off[il]]
        pres[net.lane_ctrl[l], net.lane_group[l]] += int(np.sum(counts[l] - counts[tg]))
    for c in range(net.n_ctrl):
        if cs[c, 1] >= 0:
            continue
        pr = pres[c, :net.ctrl_nphase[c]]
        best = int(np.argmax(pr))
        if pr[cs[c, 0]] == pr[best]:
            best = cs[c, 0]
        if best != cs[c, 0]:
            if net.ctrl_yellow[c] > 0:
                cs[c, 1], cs[c, 2] = best, t + net.ctrl_yellow[c]
            else:
                cs[c, 0] = best
    return cs


@pytest.mark.parametrize("interval", [10, 2])
def test_max_pressure_run_matches_brute_force_and_never_runs_red(oracle_lib, interval):
    """Small grid workload under max pressure: at every step the controllers equal R13
    restated with numpy from the previous step's controllers and the snapshot's lane
    counts; a switch starts only at a decision step and its yellow lasts exactly the
    controller's yellow time; no vehicle crosses a red stop line; all trips arrive.  With
    decisions every 2 s, shorter than the 3 s yellow, decision steps fall inside a pending
    switch, which they leave alone."""
    import oracle
    net, dem = synth.small_grid_workload(2)
    MPI = dict(MP, mp_interval=interval)
    o = oracle.Oracle(net, dem, MPI)
    prev = np.tile(np.array([0, -1, 0], np.int32), (net.n_ctrl, 1))   # the start state
    switches = 0
    for _ in range(3600):
        st = o.state()
        t = st["t"]
        cs = o.ctrl_state()   # the controllers step t uses
        act = st["status"] == 1
        counts = np.bincount(st["lane"][act], minlength=net.n_lanes)
        np.testing.assert_array_equal(cs, _mp_brute(net, counts, prev, t, interval), err_msg=f"step {t}")
        started = (cs[:, 1] >= 0) & (prev[:, 1] < 0)
        if started.any():
            assert t % interval == 0
            assert np.all(cs[started, 2] == t + net.ctrl_yellow[started])
            switches += int(started.sum())
        ctrl = net.lane_ctrl[st["lane"]]
        red = act & (ctrl >= 0) & (net.lane_edge[st["lane"]] >= 0) & \
            (net.lane_group[st["lane"]] != cs[np.maximum(ctrl, 0), 0])
        err, _ = o.step()
        assert err == 0
        nx = o.state()
        crossed = red & (nx["lane"] != st["lane"]) & (nx["status"] == 1) & (net.lane_edge[nx["lane"]] < 0)
        assert not crossed.any(), np.nonzero(crossed)[0][:5]
        prev = cs
        if (nx["status"] == 2).all():
            break
    assert switches > 10
    assert (o.state()["status"] == 2).all()


# ---------------------------------------------------------------------------------------
# lane speed limits and closures (R14)
# ---------------------------------------------------------------------------------------

def test_lane_speed_limit_caps_the_desired_speed(oracle_lib):
    """Free road under a lane limit of 8 m/s (v0 = 13.9): every step's acceleration is the
    free-road IDM value with v0 = 8, a_max (1 - (v/8)^4), so the vehicle approaches 8 m/s
    and never exceeds it (the map v + a_max (1 - (v/8)^4) is increasing on [0, 8] and fixes
    8); without the limit it passes 8 m/s."""
    import oracle
    net = netkit.line(3, 2000.0, 1)
    lane0 = int(net.edge_lane0[0])
    dem = netkit.vehicles([lane0], [30.0], [0.0], [[0, 1]])
    o = oracle.Oracle(net, dem, P)
    o.set_lane_limits([lane0], vmax=[8.0])
    for _ in range(60):
        v = o.state()["v"][0]
        _, d = o.step(debug=True)
        assert d["a_own"][0] == pytest.approx(P["idm_a"] * (1 - (v / 8.0) ** 4), abs=1e-12)
    v_lim = o.state()["v"][0]
    assert 7.9 < v_lim <= 8.0
    free = oracle.Oracle(net, dem, P)
    free.run(60)
    assert free.state()["v"][0] > 9.0


def test_mobil_uses_the_target_lanes_limit(oracle_lib):
    """Free-gain case with the target lane limited to 8 m/s: the changer's prospective
    acceleration is a_max (1 - (10/8)^4) < 0, so the incentive is that value and nobody
    changes; a closed target lane is not even a candidate."""
    v, v0 = 10.0, 13.9
    se = (P["idm_s0"] + v * P["idm_T"]) / math.sqrt(1 - (v / v0) ** 4)
    net = netkit.line(3, 300.0, 2)
    dem = netkit.vehicles([0, 0], [100.0, 100.0 + P["veh_len"] + se], [v, v], [[0, 1]] * 2, v0=v0)
    import oracle
    o = oracle.Oracle(net, dem, P)
    o.set_lane_limits([1], vmax=[8.0])
    _, d = o.step(debug=True)
    assert d["lc_cand"][0] == 1
    assert d["incentive"][0] == pytest.approx(P["idm_a"] * (1 - (v / 8.0) ** 4) - d["a_own"][0], abs=1e-9)
    assert d["lc_dir"][0] == 0
    o = oracle.Oracle(net, dem, P)
    o.set_lane_limits([1], closed=[1])
    _, d = o.step(debug=True)
    assert d["lc_cand"][0] == 0 and d["lc_dir"][0] == 0


def test_old_follower_drives_under_its_own_lanes_limit(oracle_lib):
    """Own lane limited to 8 m/s, target lane free: the changer c (8 m/s) is 10 m behind a
    stopped leader, its old follower O (8 m/s) behind it.  O's accelerations before and
    after the change take O's desired speed under the own lane's limit, min(13.9, 8) = 8.
    O 10 m behind: neither acceleration is clamped, so a desired speed taken for one of them
    alone from elsewhere would not cancel in the difference; O 2 m behind: its present
    acceleration is clamped at a_min and only its prospective one carries the free-road
    term (v/v0)^4 = 1."""
    am, b, T, s0, L, pol = P["idm_a"], P["idm_b"], P["idm_T"], P["idm_s0"], P["veh_len"], P["mobil_p"]

    def idm(v, v0, gap, vl):
        ss = s0 + max(0.0, v * T + v * (v - vl) / (2 * math.sqrt(am * b)))
        return max(am * (1 - (v / v0) ** 4 - (ss / gap) ** 2), P["a_min"])
    v0f = float(np.float32(13.9))
    net = netkit.line(3, 300.0, 2)
    import oracle
    for gO, clamped in ((10.0, False), (2.0, True)):
        dem = netkit.vehicles([0, 0, 0], [100.0, 100.0 + L + 10.0, 100.0 - L - gO], [8.0, 0.0, 8.0],
                              [[0, 1]] * 3)
        o = oracle.Oracle(net, dem, P)
        o.set_lane_limits([0], vmax=[8.0])
        _, d = o.step(debug=True)
        assert d["lc_cand"][0] == 1 and d["old_foll"][0] == 2 and d["tau_foll"][0] == -1
        a_c = idm(8.0, 8.0, 10.0, 0.0)
        a_new = am * (1 - (8.0 / v0f) ** 4)
        a_old_O, a_new_O = idm(8.0, 8.0, gO, 8.0), idm(8.0, 8.0, 10.0 + L + gO, 0.0)
        assert (a_old_O == P["a_min"]) == clamped and a_new_O > P["a_min"]
        assert d["incentive"][0] == pytest.approx(a_new - a_c + pol * (a_new_O - a_old_O), abs=1e-9), gO


def test_new_follower_drives_under_the_target_lanes_limit(oracle_lib):
    """Target lane limited to 8 m/s, own lane free: the changer c (8 m/s, 10 m behind a
    stopped leader) and a new follower F (8 m/s) 10 m behind it in the target lane.  Both of
    F's accelerations, on the free road now and behind c after the change, take F's desired
    speed under the target lane's limit, min(13.9, 8) = 8 (so the present one is 0)."""
    am, b, T, s0, L, pol = P["idm_a"], P["idm_b"], P["idm_T"], P["idm_s0"], P["veh_len"], P["mobil_p"]

    def idm(v, v0, gap, vl):
        ss = s0 + max(0.0, v * T + v * (v - vl) / (2 * math.sqrt(am * b)))
        return max(am * (1 - (v / v0) ** 4 - (ss / gap) ** 2), P["a_min"])
    v0f = float(np.float32(13.9))
    net = netkit.line(3, 300.0, 2)
    dem = netkit.vehicles([0, 0, 1], [100.0, 100.0 + L + 10.0, 100.0 - L - 10.0], [8.0, 0.0, 8.0], [[0, 1]] * 3)
    import oracle
    o = oracle.Oracle(net, dem, P)
    o.set_lane_limits([1], vmax=[8.0])
    _, d = o.step(debug=True)
    assert d["lc_cand"][0] == 1 and d["tau_foll"][0] == 2 and d["tau_lead"][0] == -1
    a_c = idm(8.0, v0f, 10.0, 0.0)
    a_new = am * (1 - (8.0 / 8.0) ** 4)
    aF_new, aF_old = idm(8.0, 8.0, 10.0, 8.0), am * (1 - (8.0 / 8.0) ** 4)
    assert aF_new > -P["mobil_bsafe"]
    assert d["incentive"][0] == pytest.approx(a_new - a_c + pol * (aF_new - aF_old), abs=1e-9)


def test_discretionary_change_only_toward_a_lane_serving_the_route(oracle_lib):
    """The middle lane of a 3-lane approach goes straight; its left neighbour serves only
    the left turn and its right neighbour only the right turn.  A vehicle heading straight
    behind a stopped leader has every reason to leave, but neither neighbour serves its next
    edge, so it is no candidate for a discretionary change on either step parity."""
    net = synth.grid_network(3, 3, 3, 300.0, green=30, yellow=3)
    e = [k for k in range(net.n_edges) if net.edge_from[k] == 3 and net.edge_to[k] == 4][0]
    ex = [k for k in range(net.n_edges) if net.edge_from[k] == 4 and net.edge_to[k] == 5][0]
    l0 = int(net.edge_lane0[e])
    serves = lambda l, f: f in net.succ_edge[net.succ_off[l]:net.succ_off[l + 1]]
    assert serves(l0 + 1, ex) and not serves(l0, ex) and not serves(l0 + 2, ex)
    import oracle
    for t0 in (0, 1):
        dem = netkit.vehicles([l0 + 1, l0 + 1], [100.0, 108.0], [5.0, 0.0], [[e, ex]] * 2)
        o = oracle.Oracle(net, dem, P)
        st = o.state()
        o.set_state(st["status"], st["lane"], st["x"], st["v"], st["rp"], t0)
        _, d = o.step(debug=True)
        assert d["lc_cand"][0] == 0 and d["lc_dir"][0] == 0, t0


def test_closed_lane_is_never_entered_until_reopened(oracle_lib):
    """A vehicle whose next edge's lanes are closed stops at the end of the lane before them
    (gap >= 0, never on a closed lane) and goes on once they reopen."""
    import oracle
    net = netkit.line(3, 300.0, 1)
    l0, l1 = int(net.edge_lane0[0]), int(net.edge_lane0[1])
    dem = netkit.vehicles([l0], [200.0], [12.0], [[0, 1]])
    o = oracle.Oracle(net, dem, P)
    o.set_lane_limits([l1], closed=[1])
    for _ in range(80):
        o.step()
        st = o.state()
        assert st["status"][0] == 1 and st["lane"][0] != l1
        ln = int(st["lane"][0])
        assert st["x"][0] <= net.lane_len[ln] + 1e-9
    assert st["v"][0] == pytest.approx(0.0, abs=1e-6)
    o.set_lane_limits([l1], closed=[0])
    o.run(120)
    assert o.state()["status"][0] == 2


def test_departures_wait_on_a_closed_lane(oracle_lib):
    import oracle
    net = netkit.line(3, 300.0, 1)
    l0 = int(net.edge_lane0[0])
    dem = netkit.vehicles([-1], [0.0], [0.0], [[0, 1]], t_dep=[0])
    o = oracle.Oracle(net, dem, P)
    o.set_lane_limits([l0], closed=[1])
    o.run(10)
    assert o.state()["status"][0] == 0
    o.set_lane_limits([l0], closed=[0])
    o.step()
    assert o.state()["status"][0] == 1


# ---------------------------------------------------------------------------------------
# whole-run invariants
# ---------------------------------------------------------------------------------------

def _check_run(o, net, n_steps, L=5.0):
    n = o.n
    st0 = o.state()
    placed = int((st0["status"] == 1).sum())
    for t in range(n_steps):
        st = o.state()
        act = st["status"] == 1
        # red lights at the start of the step
        red = np.array([o.signal_state(int(l), st["t"]) == 2 if a and net.lane_edge[l] >= 0 else False
                        for l, a in zip(st["lane"], act)])
        err, _ = o.step()
        assert err == 0
        nx = o.state()
        # no crossing on red: a vehicle on a red edge lane stays on it (or arrives if it is
        # the destination edge, whose end is open)
        crossed = red & (nx["lane"] != st["lane"]) & (nx["status"] == 1) & \
            (net.lane_edge[nx["lane"]] < 0)
        assert not crossed.any()
        # gap >= 0 in every lane
        a = np.nonzero(nx["status"] == 1)[0]
        o_ = np.lexsort((nx["x"][a], nx["lane"][a]))
        la, xa = nx["lane"][a][o_], nx["x"][a][o_]
        same = la[1:] == la[:-1]
        gaps = (xa[1:] - L - xa[:-1])[same]
        assert gaps.size == 0 or gaps.min() >= -1e-9, gaps.min()
        # conservation
        m = o.metrics()
        assert (nx["status"] == 0).sum() + (nx["status"] == 1).sum() + (nx["status"] == 2).sum() == n
        assert m["inserted"] + placed == (nx["status"] == 1).sum() + (nx["status"] == 2).sum()
        assert m["arrived"] == (nx["status"] == 2).sum()
    return o.state()


@pytest.mark.parametrize("seed", [1, 2])
def test_small_grid_run_invariants(oracle_lib, seed):
    net, dem = synth.small_grid_workload(seed)
    o = oracle_lib.Oracle(net, dem, P, n_windows=12)
    st = _check_run(o, net, 1500)
    assert (st["status"] == 2).sum() > 0.9 * dem.n


def test_delaunay_run_invariants_with_merges(oracle_lib):
    net = synth.delaunay_network(60, box=2500.0, seed=4)
    # vehicles on internal lanes feeding multi-feeder targets exercise the merge rule
    n_pred = np.bincount(net.succ_lane[net.succ_off[net.n_edge_lanes]:], minlength=net.n_lanes)
    assert (n_pred > 1).any()
    dem = synth.merge_demands(
        synth.place_vehicles(net, 400, seed=4, min_spacing=7.0, internal_frac=1.0),
        synth.uniform_trips(net, 400, 300, seed=5))
    o = oracle_lib.Oracle(net, dem, dict(P, p_lc=0.5), n_windows=2)
    _check_run(o, net, 400)


def test_run_is_deterministic_and_resumable(oracle_lib):
    net, dem = synth.small_grid_workload(3)
    a = oracle_lib.Oracle(net, dem, P, n_windows=12)
    b = oracle_lib.Oracle(net, dem, P, n_windows=12)
    a.run(700)
    b.run(300)
    s = b.state()
    c = oracle_lib.Oracle(net, dem, P, n_windows=12)
    c.set_state(s["status"], s["lane"], s["x"], s["v"], s["rp"], s["t"], s["t_arr"])
    c.run(400)
    sa, sc = a.state(), c.state()
    for k in ("status", "lane", "x", "v", "rp", "t_arr", "t"):
        np.testing.assert_array_equal(sa[k], sc[k])


def test_rewinding_a_run_resumes_it_exactly(oracle_lib):
    """A state written back into a simulation that has run past it (a rewind, with trips
    that have since departed waiting again) resumes exactly: from the state at t = 300 of
    a run that went on to t = 700, the same 400 steps lead to the same state as before."""
    net, dem = synth.small_grid_workload(3)
    a = oracle_lib.Oracle(net, dem, P)
    a.run(300)
    s = a.state()
    a.run(400)
    end = a.state()
    a.set_state(s["status"], s["lane"], s["x"], s["v"], s["rp"], s["t"], s["t_arr"])
    assert (a.state()["status"] == 0).sum() > (end["status"] == 0).sum()   # trips wait again
    a.run(400)
    again = a.state()
    for k in ("status", "lane", "x", "v", "rp", "t_arr", "t"):
        np.testing.assert_array_equal(end[k], again[k])


def test_lane_link_changes_are_checked(oracle_lib):
    """The oracle's lane-link call refuses a junction lane or a lane out of range and
    changes nothing then."""
    import oracle
    net = netkit.line(3, 300.0, 2)
    dem = netkit.vehicles([0], [100.0], [5.0], [[0, 1]])
    o = oracle.Oracle(net, dem, P)
    for bad in ([net.n_edge_lanes], [net.n_lanes], [-1]):
        with pytest.raises(ValueError):
            o.set_lane_links(bad, [0])
    o.run(60)
    assert o.state()["status"][0] == 2 or o.state()["lane"][0] != 0   # its link stayed open


def test_departures_fifo_and_room(oracle_lib):
    net = netkit.line(3, 300.0, 2)
    n = 5
    dem = netkit.vehicles([-1] * n, [0.0] * n, [0.0] * n, [[0, 1]] * n)
    o = oracle_lib.Oracle(net, dem, P)
    assert o.departure_lane(0) == 0
    order = []
    for t in range(60):
        st = o.state()
        act = np.nonzero(st["status"] == 1)[0]
        on0 = act[st["lane"][act] == 0]
        tail_x = st["x"][on0].min() if on0.size else None
        _, d = o.step(debug=True)
        ins = np.nonzero(d["inserted"])[0].tolist()
        if ins:
            assert tail_x is None or tail_x - 5.0 >= 5.0 + P["idm_s0"]
        elif tail_x is not None and len(order) < n:
            assert tail_x - 5.0 < 5.0 + P["idm_s0"]
        order += ins
    assert order == list(range(n))


def test_departure_waits_for_its_time(oracle_lib):
    """A trip enters at the step whose clock equals its departure time (on an empty lane
    there is room at once): waiting before it, inserted by it, active after it, standing
    with its whole length on the lane (front at x = L) at rest."""
    net = netkit.line(3, 300.0, 1)
    dem = netkit.vehicles([-1], [0.0], [0.0], [[0, 1]], t_dep=[5])
    o = oracle_lib.Oracle(net, dem, P)
    for t in range(8):
        assert o.state()["t"] == t
        assert o.state()["status"][0] == (0 if t <= 5 else 1), t
        _, d = o.step(debug=True)
        assert d["inserted"][0] == (1 if t == 5 else 0), t
        if t == 5:
            st = o.state()
            assert st["lane"][0] == net.edge_lane0[0] and st["x"][0] == P["veh_len"] and st["v"][0] == 0.0


def test_departures_enter_the_first_lane_linked_to_the_next_edge(oracle_lib):
    """On the 3-lane approaches of a grid (lane 0 serves only the right turn) every trip
    enters the lowest-index lane of its first edge that links to its second edge."""
    net = synth.grid_network(3, 3, 3, 300.0, green=30, yellow=3)
    trips = []
    for e in range(net.n_edges):
        l0 = int(net.edge_lane0[e])
        nxt = sorted({int(f) for q in range(int(net.edge_nlanes[e]))
                      for f in net.succ_edge[net.succ_off[l0 + q]:net.succ_off[l0 + q + 1]]})
        for f in nxt:
            want = min(l0 + q for q in range(int(net.edge_nlanes[e]))
                       if f in net.succ_edge[net.succ_off[l0 + q]:net.succ_off[l0 + q + 1]])
            trips.append(([e, f], want))
    assert any(w != int(net.edge_lane0[r[0]]) for r, w in trips)
    dem = netkit.vehicles([-1] * len(trips), [0.0] * len(trips), [0.0] * len(trips), [r for r, _ in trips],
                          t_dep=[3 * k for k in range(len(trips))])
    o = oracle_lib.Oracle(net, dem, P)
    lane_at_entry = {}
    for _ in range(3 * len(trips) + 40):
        _, d = o.step(debug=True)
        st = o.state()
        for i in np.nonzero(d["inserted"])[0]:
            lane_at_entry[int(i)] = int(st["lane"][i])
    assert len(lane_at_entry) == len(trips)
    assert all(lane_at_entry[k] == w for k, (_, w) in enumerate(trips))


def test_departure_queue_is_first_in_first_out_by_departure_time(oracle_lib):
    """Five trips on one departure lane with departure times 8, 6, 4, 2, 0 (ids in the
    opposite order) enter in the order of their departure times, each once there is room."""
    net = netkit.line(3, 300.0, 1)
    n = 5
    dem = netkit.vehicles([-1] * n, [0.0] * n, [0.0] * n, [[0, 1]] * n, t_dep=[8, 6, 4, 2, 0])
    o = oracle_lib.Oracle(net, dem, P)
    order = []
    for _ in range(80):
        _, d = o.step(debug=True)
        order += np.nonzero(d["inserted"])[0].tolist()
    assert order == [4, 3, 2, 1, 0]


def test_departure_room_counts_the_arrivals_of_the_step(oracle_lib):
    """A vehicle crossing from a junction lane onto a departure lane lands 11 m in, so its
    rear is 6 m from the lane start, less than L + s0 = 7 m: the departure due at that step
    waits; at the next step the same vehicle, now the lane's rearmost in the snapshot, still
    leaves no room; one step later it has moved on and the departure enters."""
    net = netkit.line(4, 300.0, 1)
    l0, l1 = int(net.edge_lane0[0]), int(net.edge_lane0[1])
    il = int(net.succ_lane[net.succ_off[l0]])
    assert int(net.succ_lane[net.succ_off[il]]) == l1
    v, v0 = 12.0, 13.9
    a = P["idm_a"] * (1 - (v / float(np.float32(v0))) ** 4)     # free road (nothing ahead)
    d_step = 0.5 * (v + v + a * P["dt"]) * P["dt"]
    x = float(net.lane_len[il]) - (d_step - 11.0)
    dem = netkit.vehicles([il, -1], [x, 0.0], [v, 0.0], [[0, 1, 2], [1, 2]], v0=v0, t_dep=[0, 0])
    o = oracle_lib.Oracle(net, dem, P)
    assert o.departure_lane(1) == l1
    _, d = o.step(debug=True)
    st = o.state()
    assert st["lane"][0] == l1 and st["x"][0] == pytest.approx(11.0, abs=1e-5)
    assert d["inserted"][1] == 0 and st["status"][1] == 0
    _, d = o.step(debug=True)
    assert d["inserted"][1] == 0
    assert o.state()["x"][0] - P["veh_len"] >= P["veh_len"] + P["idm_s0"]
    _, d = o.step(debug=True)
    assert d["inserted"][1] == 1


def test_travel_time_is_the_arrival_clock_minus_the_departure(oracle_lib):
    """Trip travel times counted by the oracle against the clock seen from outside: a trip
    that finishes during the step at clock t arrives at t + 1, and the summed travel time
    is the sum over arrived trips of that arrival clock minus the departure time."""
    net, dem = synth.small_grid_workload(2)
    o = oracle_lib.Oracle(net, dem, P)
    arrive = {}
    for _ in range(900):
        before = o.state()
        o.step()
        after = o.state()
        for i in np.nonzero((after["status"] == 2) & (before["status"] != 2))[0]:
            arrive[int(i)] = after["t"]
    assert len(arrive) > 50
    st = o.state()
    assert all(st["t_arr"][i] == t for i, t in arrive.items())
    m = o.metrics()
    assert m["arrived"] == len(arrive)
    assert m["sum_tt"] == sum(t - int(dem.t_dep[i]) for i, t in arrive.items())


def test_metrics_window_sums(oracle_lib):
    net, dem = synth.small_grid_workload(1)
    o = oracle_lib.Oracle(net, dem, dict(P, window=50), n_windows=4)
    vs = np.zeros((4, net.n_lanes))
    vc = np.zeros((4, net.n_lanes), np.int64)
    for t in range(200):
        st = o.state()
        a = st["status"] == 1
        np.add.at(vs[t // 50], st["lane"][a], st["v"][a])
        np.add.at(vc[t // 50], st["lane"][a], 1)
        o.step()
    m = o.metrics()
    np.testing.assert_array_equal(m["vcnt"], vc)
    np.testing.assert_allclose(m["vsum"], vs, rtol=1e-12)


def test_mobil_politeness_terms_closed_form(oracle_lib):
    """Stopped followers make every IDM term closed-form: at v = 0, s* = s0 and
    a = a_max (1 - (s0/s)^2).  New follower F 10 m behind in the target lane, old follower
    O 4 m behind in the own lane; the changer c follows its leader at equilibrium."""
    v, v0 = 10.0, 13.9
    v0f = float(np.float32(v0))
    se = (P["idm_s0"] + v * P["idm_T"]) / math.sqrt(1 - (v / v0) ** 4)
    xc, L, s0, am = 100.0, P["veh_len"], P["idm_s0"], P["idm_a"]
    gF, gO = 10.0, 4.0
    d = _two_lane_case([0, 0, 1, 0], [xc, xc + L + se, xc - L - gF, xc - L - gO], [v, v, 0.0, 0.0])
    assert d["tau_foll"][0] == 2 and d["old_foll"][0] == 3 and d["tau_lead"][0] == -1
    free_gain = am * (1 - (v / v0f) ** 4)
    dF = am * (1 - (s0 / gF) ** 2) - am            # F: free road -> behind c
    gO_new = gO + L + se                           # O: behind c -> behind c's leader
    dO = am * (1 - (s0 / gO_new) ** 2) - am * (1 - (s0 / gO) ** 2)
    want = free_gain + P["mobil_p"] * (dF + dO)
    assert d["incentive"][0] == pytest.approx(want, abs=1e-5)
    assert d["lc_dir"][0] == +1


def test_level_vehicle_in_the_target_lane_is_the_follower(oracle_lib):
    """A target-lane vehicle exactly level with the changer (same x) is its new follower,
    not its leader (the leader is the first with x' > x): it sits at gap -L behind the
    changer, so the conflict guard rejects the change."""
    d = _two_lane_case([0, 0, 1, 1], [100.0, 108.0, 100.0, 130.0], [5.0, 0.0, 5.0, 5.0])
    assert d["lc_cand"][0] == 1
    assert d["tau_foll"][0] == 2 and d["tau_lead"][0] == 3
    assert d["lc_dir"][0] == 0


def test_mobil_politeness_with_a_target_leader(oracle_lib):
    """Everybody stopped (v = 0: s* = s0, a = a_max (1 - (s0/s)^2) whatever the leader
    does): the changer c 2.5 m behind its own leader, a target leader 3 m ahead of it and a
    new follower F 3 m behind it in the target lane.  F's old gap runs to the target leader
    (3 + L + 3 m); its new gap is the 3 m to c."""
    xc, L, s0, am = 100.0, P["veh_len"], P["idm_s0"], P["idm_a"]
    d = _two_lane_case([0, 0, 1, 1], [xc, xc + L + 2.5, xc + L + 3.0, xc - L - 3.0], [0.0] * 4)
    assert d["tau_lead"][0] == 2 and d["tau_foll"][0] == 3 and d["old_foll"][0] == -1
    idm0 = lambda gap: am * (1 - (s0 / gap) ** 2)
    want = idm0(3.0) - idm0(2.5) + P["mobil_p"] * (idm0(3.0) - idm0(3.0 + L + 3.0))
    assert d["a_own"][0] == pytest.approx(idm0(2.5), abs=1e-12)
    assert d["incentive"][0] == pytest.approx(want, abs=1e-9)
    assert d["lc_dir"][0] == (+1 if want > P["mobil_th"] else 0)


def test_merge_projection_leader(oracle_lib):
    """Two internal lanes feeding one exit lane: the vehicle farther from the merge point
    follows the projected rear of the nearer one (gap = d_A - d_B - L); the nearer one
    does not see the farther one; on equal distance the lower id goes first."""
    net = synth.grid_network(3, 3, 1, 300.0, green=30, yellow=3)
    nel = net.n_edge_lanes
    tgt = net.succ_lane[net.succ_off[nel:net.n_lanes]]
    counts = np.bincount(tgt, minlength=net.n_lanes)
    lt = int(np.nonzero(counts >= 2)[0][0])
    f1, f2 = [nel + int(i) for i in np.nonzero(tgt == lt)[0][:2]]
    appr = {}
    for l in range(nel):
        for k in range(net.succ_off[l], net.succ_off[l + 1]):
            appr[int(net.succ_lane[k])] = int(net.lane_edge[l])
    ex = int(net.lane_edge[lt])

    def case(dA, dB):
        xs = [net.lane_len[f1] - dA, net.lane_len[f2] - dB]
        dem = netkit.vehicles([f1, f2], xs, [3.0, 3.0], [[appr[f1], ex], [appr[f2], ex]])
        o = oracle_lib.Oracle(net, dem, P)
        st = o.state()
        o.set_state(st["status"], st["lane"], st["x"], st["v"], st["rp"], 0)
        _, d = o.step(debug=True)
        return d
    d = case(10.0, 4.0)
    assert d["lead_id"][0] == 1 and d["s_own"][0] == pytest.approx(10.0 - 4.0 - P["veh_len"], abs=1e-5)
    assert d["lead_id"][1] == -1
    d = case(6.0, 6.0)          # tie: id 0 goes first, id 1 follows at gap -L
    assert d["lead_id"][0] == -1
    assert d["lead_id"][1] == 0 and d["s_own"][1] == pytest.approx(-P["veh_len"], abs=1e-5)


# ---------------------------------------------------------------------------------------
# dynamic lanes (R17)
# ---------------------------------------------------------------------------------------

def test_closed_links_force_the_mandatory_change(oracle_lib):
    """Straight road, 2 lanes: with its links open a lone vehicle stays on lane 0 (empty
    neighbour, zero incentive); with lane 0's links closed lane 0 no longer leads to the
    next edge, so at the even step (moves toward higher lane index allowed) it changes to
    lane 1 at once."""
    import oracle
    net = netkit.line(3, 300.0, 2)
    l0 = int(net.edge_lane0[0])
    dem = netkit.vehicles([l0], [100.0], [10.0], [[0, 1]])
    a = oracle.Oracle(net, dem, P)
    a.step()
    assert a.state()["lane"][0] == l0
    b = oracle.Oracle(net, dem, P)
    b.set_lane_links([l0], [0])
    _, d = b.step(debug=True)
    assert d["lc_dir"][0] == 1 and b.state()["lane"][0] == l0 + 1


def test_closed_link_moves_the_fan_out_choice(oracle_lib):
    """Lane 0 of the first edge links to the next edge twice (two internal lanes, CSR
    order); a vehicle crossing the junction takes the first, or the second once the first
    is closed, and the first again once it reopens."""
    import oracle
    net = netkit.line(3, 300.0, 2)
    l0 = int(net.edge_lane0[0])
    first, second = (int(net.succ_lane[k]) for k in range(net.succ_off[l0], net.succ_off[l0] + 2))
    dem = netkit.vehicles([l0], [296.0], [10.0], [[0, 1]])
    for mask, want in ((0b11, first), (0b10, second), (0b01, first)):
        o = oracle.Oracle(net, dem, P)
        o.set_lane_links([l0], [mask])
        o.step()
        assert o.state()["lane"][0] == want, (mask, o.state()["lane"][0])


def test_all_open_links_change_nothing(oracle_lib):
    """Opening every link of every edge lane (their state at load) leaves a whole run
    bit-identical."""
    import oracle
    net, dem = synth.small_grid_workload(3)
    a = oracle.Oracle(net, dem, P)
    b = oracle.Oracle(net, dem, P)
    el = np.nonzero(net.lane_edge >= 0)[0]
    b.set_lane_links(el, (1 << np.diff(net.succ_off)[el]) - 1)
    a.run(600)
    b.run(600)
    sa, sb = a.state(), b.state()
    for k in ("status", "lane", "x", "v", "rp"):
        np.testing.assert_array_equal(sa[k], sb[k])


def test_max_pressure_skips_closed_links(oracle_lib):
    """Small grid under max pressure with 30% of the closable links closed: at every step
    the controllers equal R13 restated with numpy over the open links only."""
    import oracle
    net, dem = synth.small_grid_workload(2)
    mask = netkit.closable_links(net, dem, np.random.default_rng(4), 0.3)
    closed = {(l, j) for l, m in mask.items() for j in range(int(net.succ_off[l + 1] - net.succ_off[l]))
              if not (m >> j) & 1}
    assert len(closed) > 20
    o = oracle.Oracle(net, dem, MP)
    o.set_lane_links(list(mask), list(mask.values()))

    def brute(counts, cs_prev, t):
        cs = cs_prev.copy()
        for c in range(net.n_ctrl):
            if cs[c, 1] >= 0 and t >= cs[c, 2]:
                cs[c, 0], cs[c, 1] = cs[c, 1], -1
        if t % MP["mp_interval"]:
            return cs
        pres = np.zeros((net.n_ctrl, int(net.ctrl_nphase.max())), np.int64)
        for l in np.nonzero((net.lane_ctrl >= 0) & (net.lane_edge >= 0))[0]:
            for j, k in enumerate(range(net.succ_off[l], net.succ_off[l + 1])):
                if (int(l), j) in closed:
                    continue
                tg = net.succ_lane[net.succ_off[net.succ_lane[k]]]
                pres[net.lane_ctrl[l], net.lane_group[l]] += int(counts[l] - counts[tg])
        for c in range(net.n_ctrl):
            if cs[c, 1] >= 0:
                continue
            pr = pres[c, :net.ctrl_nphase[c]]
            best = int(np.argmax(pr))
            if pr[cs[c, 0]] == pr[best]:
                best = cs[c, 0]
            if best != cs[c, 0]:
                if net.ctrl_yellow[c] > 0:
                    cs[c, 1], cs[c, 2] = best, t + net.ctrl_yellow[c]
                else:
                    cs[c, 0] = best
        return cs

    prev = np.tile(np.array([0, -1, 0], np.int32), (net.n_ctrl, 1))
    differs = 0
    for _ in range(1200):
        st = o.state()
        cs = o.ctrl_state()
        act = st["status"] == 1
        counts = np.bincount(st["lane"][act], minlength=net.n_lanes)
        np.testing.assert_array_equal(cs, brute(counts, prev, st["t"]), err_msg=f"step {st['t']}")
        differs += int((cs != _mp_brute(net, counts, prev, st["t"], MP["mp_interval"])).any())
        prev = cs
        err, _ = o.step()
        assert err == 0
    assert differs > 0   # the closed links changed some decision
