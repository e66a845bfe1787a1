"""Pins of the oracle's learned lane change (reading R19) and of its BF16 network.

The learned form replaces the MOBIL incentive test of safe discretionary candidates by a
16 -> 64 -> 64 -> 3 network run in BF16 with FP32 accumulation (the paper's lane-change
model is rule-based, Sec. III-A; the surrogate is this library's addition).  These tests pin
the oracle's side of it against things other than itself:
  - BF16 rounding against values that follow from the format (8 significant bits, round
    to nearest, ties to even);
  - the BF16 forward against the plain FP64 forward where no value needs rounding;
  - the in-step decision against closed forms: probe networks whose decision is a known
    step function of one physical quantity (speed, distance to the lane end, own gap), a
    network that always stays, and the full-fallback network, which must reproduce the
    rule step bit for bit over a whole run.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2405_12520_b300 import synth

P = synth.default_params()


# --- BF16 rounding ------------------------------------------------------------------

# value -> nearest BF16 (8 significant bits).  Around 1 the spacing is 2^-7: 1 + 2^-8 is
# halfway between 1 and 1 + 2^-7 and goes to the even significand (1); 1 + 3 * 2^-8 is
# halfway between 1 + 2^-7 and 1 + 2^-6 and goes to 1 + 2^-6.  0.1 = 1.6 * 2^-4 and
# 1.6 * 128 = 204.8 -> 205, so 205 / 128 / 16.  Around 256 the spacing is 2: 257 -> 256 and
# 259 -> 260 (ties to even), 258 is exact.  pi: 3.14159 / 2 * 128 = 201.06 -> 201 -> 3.140625.
GOLDEN = [(1.0 + 2.0 ** -8, 1.0), (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6), (0.1, 205.0 / 128 / 16),
          (257.0, 256.0), (259.0, 260.0), (258.0, 258.0), (-3.14159, -3.140625),
          (1.0 + 2.0 ** -8 + 2.0 ** -20, 1.0 + 2.0 ** -7), (0.0, 0.0), (-0.75, -0.75)]


@pytest.mark.parametrize("x,want", GOLDEN)
def test_bf16_rounding_follows_the_format(x, want):
    assert oracle.bf16(x) == want
    assert mlp.bf16(np.array([x]))[0] == want


def test_bf16_forward_equals_plain_forward_when_nothing_rounds():
    """Small integer weights and inputs, halves as biases: every value of the network is
    exactly representable in BF16, so rounding changes nothing and the BF16 forward must
    equal the plain FP64 forward exactly."""
    rng = np.random.default_rng(0)
    p = {"W1": rng.integers(-2, 3, (64, 16)).astype(float), "b1": rng.integers(-2, 3, 64) * 0.5,
         "W2": rng.integers(-1, 2, (64, 64)).astype(float) / 4, "b2": rng.integers(-2, 3, 64) * 0.5,
         "W3": rng.integers(-1, 2, (3, 64)).astype(float) / 8, "b3": np.array([0.5, -0.5, 0.0])}
    theta = mlp.pack(p)
    X = rng.integers(-3, 4, (200, 16)).astype(float) / 4
    z, near, _ = mlp.forward_bf16(theta, X)
    z0, (_, a1, h1, a2, h2) = mlp.forward(theta, X)
    # integer inputs/weights keep h1 in quarters below 2^6 and h2 in sixteenths: exact in BF16
    assert np.array_equal(mlp.bf16(h1), h1) and np.array_equal(mlp.bf16(h2), h2)
    assert np.array_equal(z, z0)


def test_bf16_forward_rounds_where_the_kernel_rounds():
    """A network that triples input 0 through a single path: an input of 1 + 3 * 2^-9 is
    rounded to 1 + 2^-7 on entry (kept unrounded, 3 * (1 + 3 * 2^-9) = 3.017578125 would
    round to 3.015625), and the hidden value 3 * (1 + 2^-7) = 3.0234375, halfway between
    3.015625 and 3.03125 (8 significant bits), is rounded to the even 3.03125 before the next
    layer (kept, the logit would be 3.0234375)."""
    p = {k: np.zeros(s) for k, s in mlp.SHAPES}
    p["W1"][0, 0] = 3.0
    p["W2"][0, 0] = 1.0
    p["W3"][1, 0] = 1.0
    theta = mlp.pack(p)
    X = np.zeros((1, 16))
    X[0, 0] = 1.0 + 3 * 2.0 ** -9
    z, _, _ = mlp.forward_bf16(theta, X)
    assert z[0, 1] == 3.03125 and z[0, 0] == 0.0 and z[0, 2] == 0.0


# --- the in-step learned decision ----------------------------------------------------

def _workload():
    net = synth.grid_network(6, 6, 3, 300.0, 30, 3, "wave")
    dem = synth.merge_demands(synth.place_vehicles(net, 2500, seed=41, min_spacing=7.0, internal_frac=0.2),
                              synth.uniform_trips(net, 300, 30, seed=42))
    return net, dem


def _probe(k: int, theta_k: float, G: float = 256.0, K: float = 16.0):
    """Probe network: change lane in the step's allowed direction when input k is at least
    theta_k + 1/G, stay when it is at most theta_k.  Layer 1: q = relu(1 + G (theta_k - f_k)),
    u = relu(f5), w = relu(-f5) (f5 = allowed direction); layer 2: s_l = relu(u - q),
    s_r = relu(w - q) (q = 0 past the threshold, >= 1 below it); logits (K/2, K s_l, K s_r):
    softmax margin 0.9993 either way."""
    p = {k_: np.zeros(s) for k_, s in mlp.SHAPES}
    p["W1"][0, k] = -G
    p["b1"][0] = 1.0 + G * theta_k
    p["W1"][1, 5] = 1.0
    p["W1"][2, 5] = -1.0
    p["W2"][0, 1] = 1.0
    p["W2"][0, 0] = -1.0
    p["W2"][1, 2] = 1.0
    p["W2"][1, 0] = -1.0
    p["W3"][1, 0] = K
    p["W3"][2, 1] = K
    p["b3"][0] = K / 2
    return mlp.pack(p).astype(np.float32)


def _pair(net, dem, t0, theta, margin=0.2):
    """The same state stepped once by the rule and by the learned oracle, with records."""
    rule = oracle.Oracle(net, dem, P)
    lrn = oracle.Oracle(net, dem, P)
    lrn.set_lc_model(theta, margin)
    st = rule.state()
    for o in (rule, lrn):
        o.set_state(st["status"], st["lane"], st["x"], st["v"], st["rp"], t0, st["t_arr"])
    _, dr = rule.step(debug=True)
    _, dl = lrn.step(debug=True)
    return st, dr, dl


@pytest.mark.parametrize("t0", [0, 1])
def test_learned_always_stay_network_removes_only_discretionary_changes(t0):
    p = {k: np.zeros(s) for k, s in mlp.SHAPES}
    p["b3"][0] = 8.0
    theta = mlp.pack(p).astype(np.float32)
    net, dem = _workload()
    st, dr, dl = _pair(net, dem, t0, theta)
    act = dr["active_before"] == 1
    L = dl["lc_learn"] == 1
    assert L.sum() > 50, L.sum()
    assert np.all(dr["lc_cand"][L] == 1)            # the network decides candidates only
    assert np.all(dl["lc_dir"][L] == 0)              # ... and always says stay
    assert (dr["lc_dir"][L] != 0).sum() > 0          # the rule would have changed some
    rest = act & ~L                                  # mandatory changes and all others: the rule's
    assert np.array_equal(dl["lc_dir"][rest], dr["lc_dir"][rest])
    assert np.all(dl["lc_margin"][L] > 0.99)
    assert np.all(dl["flag"][L] == dr["flag"][L])    # far from the margin: no new flags


@pytest.mark.parametrize("k,theta_k,quantity,lo,hi", [
    (0, 0.5, "speed", 9.8, 10.3),               # input 0 = v / 20: change above 10 m/s
    (13, 1.0, "to_end", 98.0, 102.0),           # input 13 = min(len - x, 200) / 100
    (2, 0.25, "gap", 24.5, 25.6),               # input 2 = min(own gap, 200) / 100, 2 if free
])
@pytest.mark.parametrize("t0", [0, 1])
def test_probe_network_decides_by_one_physical_quantity(k, theta_k, quantity, lo, hi, t0):
    net, dem = _workload()
    st, dr, dl = _pair(net, dem, t0, _probe(k, theta_k))
    L = np.nonzero(dl["lc_learn"] == 1)[0]
    assert L.size > 50
    step_dir = 1 if t0 % 2 == 0 else -1
    if quantity == "speed":
        q = st["v"][L]
    elif quantity == "to_end":
        q = np.asarray(net.lane_len, np.float64)[st["lane"][L]] - st["x"][L]
    else:
        q = np.where(dl["lead_kind"][L] == 0, np.inf, dl["s_own"][L])
    up, down = q > hi, q < lo
    assert up.sum() > 5 and down.sum() > 5, (up.sum(), down.sum())
    assert np.all(dl["lc_dir"][L[up]] == step_dir)
    assert np.all(dl["lc_dir"][L[down]] == 0)
    # the inputs the oracle recorded are the quantity in the stated scale
    f = dl["lc_feat"][L, k]
    scale = {"speed": q / 20.0, "to_end": np.minimum(q, 200.0) / 100.0,
             "gap": np.where(np.isinf(q), 2.0, np.minimum(q, 200.0) / 100.0)}[quantity]
    np.testing.assert_allclose(f, scale, rtol=1e-12, atol=1e-12)


def test_full_fallback_network_is_the_rule_over_a_run():
    """Margin 1: every learned candidate falls back to the rule, so a 400-step run with the
    learned form must give the rule's run bit for bit."""
    net, dem = synth.small_grid_workload(5)
    theta = (mlp.init(3) * 1e-3).astype(np.float32)
    rule = oracle.Oracle(net, dem, P)
    lrn = oracle.Oracle(net, dem, P)
    lrn.set_lc_model(theta, 1.0)
    n_learn = 0
    for k in range(400):
        _, _ = rule.step()
        _, dl = lrn.step(debug=(k % 50 == 0))
        if dl is not None:
            n_learn += int((dl["lc_learn"] == 1).sum())
    a, b = rule.state(), lrn.state()
    for key in ("status", "lane", "x", "v", "rp", "t_arr"):
        assert np.array_equal(a[key], b[key]), key
    assert n_learn > 0


def test_learned_logits_match_the_numpy_bf16_forward():
    """The C oracle's network and oracle/mlp.forward_bf16 (the same BF16 rounding points)
    agree on every learned candidate of a step: two restatements of one definition."""
    net, dem = _workload()
    theta = (mlp.init(5) + np.random.default_rng(1).normal(scale=0.05, size=mlp.N_PARAMS)).astype(np.float32)
    st, dr, dl = _pair(net, dem, 0, theta, margin=0.0)
    L = np.nonzero(dl["lc_learn"] == 1)[0]
    z, _, _ = mlp.forward_bf16(theta.astype(np.float64), dl["lc_feat"][L])
    np.testing.assert_allclose(dl["lc_logit"][L], z, rtol=1e-12, atol=1e-12)
    mg, cls = mlp.margin_class(z)
    np.testing.assert_allclose(dl["lc_margin"][L], mg, rtol=1e-12, atol=1e-12)
    # margin 0: the class decides; at t0 = 0 only left is allowed, so right means stay
    assert np.array_equal(dl["lc_dir"][L], np.where(cls == 1, 1, 0))
    assert (cls == 1).sum() > 0 and (cls != 1).sum() > 0


@pytest.mark.parametrize("t0", [0, 1])
def test_always_right_network_changes_only_on_right_steps(t0):
    """A network that always answers 'right' (class 2, margin 0.9993): on a step that allows
    only moves to the left (even t) every learned candidate stays; on a step that allows
    moves to the right (odd t) every learned candidate moves right, since it passed the
    safety criteria for that target lane and the class replaces the incentive test."""
    p = {k: np.zeros(s) for k, s in mlp.SHAPES}
    p["b3"][2] = 8.0
    theta = mlp.pack(p).astype(np.float32)
    net, dem = _workload()
    st, dr, dl = _pair(net, dem, t0, theta)
    act = dr["active_before"] == 1
    L = dl["lc_learn"] == 1
    assert L.sum() > 50, L.sum()
    assert np.all(dl["lc_dir"][L] == (0 if t0 % 2 == 0 else -1))
    assert np.array_equal(dl["lc_dir"][act & ~L], dr["lc_dir"][act & ~L])


@pytest.mark.parametrize("t0", [0, 1])
def test_learned_inputs_follow_from_the_state(t0):
    """The inputs of every learned candidate recomputed from the state arrays and the
    sensing records (own leader, target-lane leader and follower, old follower, whose ids the
    oracle's brute-force pins fix), in the scales of the learned decision's definition:
    speeds / 20, gaps and the distance to the lane end min(., 200) / 100 (2 when there is
    nothing), closing speeds / 10, accelerations / a_max, the step's direction."""
    net, dem = _workload()
    theta = (mlp.init(5) + np.random.default_rng(1).normal(scale=0.05, size=mlp.N_PARAMS)).astype(np.float32)
    st, dr, dl = _pair(net, dem, t0, theta, margin=0.0)
    L = np.nonzero(dl["lc_learn"] == 1)[0]
    assert L.size > 50
    f = dl["lc_feat"][L]
    x, v, lane = st["x"], st["v"], st["lane"]
    Lv = P["veh_len"]
    lane_len = np.asarray(net.lane_len, np.float64)
    v0 = np.asarray(dem.v0, np.float32).astype(np.float64)
    cap = lambda g: np.minimum(g, 200.0) / 100.0
    ok = lambda a, b: np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    ok(f[:, 0], v[L] / 20.0)
    ok(f[:, 1], v0[L] / 20.0)
    kind, s_own, vl = dl["lead_kind"][L], dl["s_own"][L], dl["vl_own"][L]
    assert set(np.unique(kind)) <= {0, 1, 2}
    ok(f[:, 2], np.where(kind == 0, 2.0, cap(s_own)))
    ok(f[:, 3], np.where(kind == 1, (v[L] - vl) / 10.0, np.where(kind == 2, v[L] / 10.0, 0.0)))
    ok(f[:, 4], dl["a_own"][L] / P["idm_a"])
    ok(f[:, 5], np.full(L.size, 1.0 if t0 % 2 == 0 else -1.0))
    tl, tf, of = dl["tau_lead"][L], dl["tau_foll"][L], dl["old_foll"][L]
    to_end = lane_len[lane[L]] - x[L]
    h = tl >= 0
    ok(f[h, 6], cap(x[tl[h]] - x[L[h]] - Lv))
    ok(f[h, 7], (v[L[h]] - v[tl[h]]) / 10.0)
    # no target leader: free road (2, 0) or the target lane's end as a stopped obstacle
    free = (f[:, 6] == 2.0) & (f[:, 7] == 0.0)
    obst = np.isclose(f[:, 6], cap(to_end), rtol=1e-12, atol=1e-12) & np.isclose(
        f[:, 7], v[L] / 10.0, rtol=1e-12, atol=1e-12)
    assert np.all((free | obst)[~h])
    h = tf >= 0
    ok(f[h, 8], cap(x[L[h]] - x[tf[h]] - Lv))
    ok(f[h, 9], v[tf[h]] / 20.0)
    ok(f[~h, 8], 2.0)
    ok(f[~h, 9], 0.0)
    ok(f[~h, 10], 0.0)
    # the new follower's acceleration behind the changer, / a_max (IDM, R1, at its own speed
    # and desired speed, the changer as its leader)
    am, b, T, s0 = P["idm_a"], P["idm_b"], P["idm_T"], P["idm_s0"]
    vF, vc = v[tf[h]], v[L[h]]
    gF = x[L[h]] - x[tf[h]] - Lv
    ss = s0 + np.maximum(0.0, vF * T + vF * (vF - vc) / (2 * np.sqrt(am * b)))
    aF = np.maximum(am * (1 - (vF / v0[tf[h]]) ** 4 - (ss / np.maximum(gF, 0.01)) ** 2), P["a_min"])
    ok(f[h, 10], aF / am)
    # the changer's prospective acceleration on the target lane, / a_max: behind the target
    # leader, before the target lane's end as a stopped obstacle, or on the free road
    vv = v[L]
    v0c = v0[L]

    def idm(vx, v0x, gap, vl):
        ssx = s0 + np.maximum(0.0, vx * T + vx * (vx - vl) / (2 * np.sqrt(am * b)))
        return np.maximum(am * (1 - (vx / v0x) ** 4 - (ssx / np.maximum(gap, 0.01)) ** 2), P["a_min"])
    h = tl >= 0
    gap_t = np.where(h, x[np.maximum(tl, 0)] - x[L] - Lv, to_end)
    vl_t = np.where(h, v[np.maximum(tl, 0)], 0.0)
    a_new = np.where(h | obst & ~free, idm(vv, v0c, gap_t, vl_t), am * (1 - (vv / v0c) ** 4))
    ok(f[:, 11], a_new / am)
    h = of >= 0
    ok(f[h, 12], v[of[h]] / 20.0)
    ok(f[h, 15], cap(x[L[h]] - x[of[h]] - Lv))
    ok(f[~h, 12], 0.0)
    ok(f[~h, 15], 2.0)
    ok(f[:, 13], cap(to_end))
    ok(f[:, 14], np.where(kind == 1, vl / 20.0, np.where(kind == 2, 0.0, 1.0)))
    # every branch above was taken
    assert (tl >= 0).any() and (tl < 0).any() and (tf >= 0).any() and (tf < 0).any()
    assert (of >= 0).any() and (of < 0).any() and (kind == 1).any()


def _sparse_exact_net(rng):
    """Each hidden unit reads one input (layer 1) or two units (layer 2) with dyadic
    weights, so inputs in quarters give every activation exactly in BF16."""
    p = {k: np.zeros(s) for k, s in mlp.SHAPES}
    for j in range(64):
        p["W1"][j, j % 16] = rng.choice([-1.0, -0.5, 0.5, 1.0])
        p["W2"][j, (7 * j) % 64] = rng.choice([-0.5, 0.5, 1.0])
        p["W2"][j, (3 * j + 1) % 64] = rng.choice([-0.25, 0.25])
    p["b1"] = rng.integers(-2, 3, 64) * 0.25
    p["b2"] = rng.integers(-2, 3, 64) * 0.125
    p["W3"] = rng.integers(-2, 3, (3, 64)) * 0.25
    p["b3"] = np.array([0.25, -0.25, 0.0])
    return mlp.pack(p)


def test_bf16_gradient_is_the_plain_gradient_at_bf16_resolution():
    """Weights, inputs and activations exactly representable in BF16: the BF16 gradient then
    differs from the plain FP64 gradient (pinned by central differences) only by the BF16
    rounding of the output and hidden-layer gradients (relative 2^-9 each), far below what a
    missing, extra or transposed term would change."""
    rng = np.random.default_rng(3)
    theta = _sparse_exact_net(rng)
    X = rng.integers(-3, 4, (256, 16)).astype(float) / 4
    _, (_, _, h1, _, h2) = mlp.forward(theta, X)
    assert np.array_equal(mlp.bf16(h1), h1) and np.array_equal(mlp.bf16(h2), h2)
    y = rng.integers(0, 3, 256)
    w = np.array([1.0, 2.0, 1.5])
    ga = mlp.grad_bf16(theta, X, y, w)
    gb = mlp.grad(theta, X, y, w)
    scale = np.abs(gb).max()
    assert scale > 1e-2
    np.testing.assert_allclose(ga, gb, rtol=1e-2, atol=2e-3 * scale)
    assert np.linalg.norm(ga - gb) <= 1e-2 * np.linalg.norm(gb)


def test_bf16_gradient_rounds_the_output_gradient():
    """A class weight of 1 leaves p - onehot = 1/3 and -2/3, which are not BF16 values: the
    weight gradient of the last layer must use their BF16 roundings (0.333984375 and
    -0.66796875) while the output bias gradient keeps the exact thirds."""
    p = {k: np.zeros(s) for k, s in mlp.SHAPES}
    p["W1"][0, 0] = 1.0
    p["W2"][0, 0] = 1.0
    theta = mlp.pack(p)
    X = np.zeros((1, 16))
    X[0, 0] = 1.0
    g = mlp.unpack(mlp.grad_bf16(theta, X, np.array([0]), np.ones(3)))
    assert g["W3"][0, 0] == mlp.bf16(-2.0 / 3.0) == -0.66796875
    assert g["W3"][1, 0] == mlp.bf16(1.0 / 3.0) == 0.333984375
    np.testing.assert_allclose(g["b3"], [-2.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0], rtol=1e-15)


def test_bf16_gradient_rounds_the_hidden_gradient():
    """Uniform outputs (logits all 0) and a last layer whose column 0 is (0, 1, 1/2): the
    gradient reaching hidden unit 0 is 1/3 + 1/6 in BF16 output gradients, 0.333984375 +
    0.1669921875 = 0.5009765625 = (1 + 2^-9) / 2, which is not a BF16 value; the kernel's
    operand for the weight gradient of layer 2 is its rounding, 0.5, so dW2[0, 0] = 0.5 h1
    with h1 = 1."""
    p = {k: np.zeros(s) for k, s in mlp.SHAPES}
    p["W1"][0, 0] = 1.0
    p["W2"][0, 0] = 1.0
    p["W3"][1, 0] = 1.0
    p["W3"][2, 0] = 0.5
    p["b3"][1] = -1.0
    p["b3"][2] = -0.5
    theta = mlp.pack(p)
    X = np.zeros((1, 16))
    X[0, 0] = 1.0
    z, _, _ = mlp.forward_bf16(theta, X)
    assert np.array_equal(z, np.zeros((1, 3)))
    g = mlp.unpack(mlp.grad_bf16(theta, X, np.array([0]), np.ones(3)))
    assert mlp.bf16(0.5009765625) == 0.5
    assert g["W2"][0, 0] == 0.5



def test_flag_rule_rounds_a_boundary_value_the_other_way():
    """The flag rule of the learned decision (oracle/mlp.flip_sensitivity) on a hand-built
    network: input 1 + 3 * 2^-9 enters as 1 + 2^-7, and the hidden value 3 (1 + 2^-7) =
    3.0234375 lies exactly halfway between the BF16 neighbours 3.015625 and 3.03125, so it is
    flagged and rounded the other way alone: logit 1 moves from 3.03125 to 3.015625 (2^-6),
    which the logit bound gains on top of the last layer's accumulation bound, and the margin
    moves by the matching softmax difference; the decision changes only when the fallback
    threshold lies between the two margins.  With input 1 nothing lies near a boundary."""
    p = {k: np.zeros(s) for k, s in mlp.SHAPES}
    p["W1"][0, 0] = 3.0
    p["W2"][0, 0] = 1.0
    p["W3"][1, 0] = 1.0
    theta = mlp.pack(p)
    X = np.zeros((2, 16))
    X[0, 0] = 1.0 + 3 * 2.0 ** -9
    X[1, 0] = 1.0
    u = 2.0 ** -22
    z, m, c, zb, msens, changed = mlp.flip_sensitivity(theta, X, 0.2)
    assert np.array_equal(z, [[0.0, 3.03125, 0.0], [0.0, 3.0, 0.0]]) and np.array_equal(c, [1, 1])
    marg = lambda l1: (np.exp(l1) - 1.0) / (np.exp(l1) + 2.0)     # softmax p1 - p0 at (0, l1, 0)
    np.testing.assert_allclose(m, [marg(3.03125), marg(3.0)], rtol=1e-12)
    acc = lambda l1: 65 * u * np.array([0.0, l1, 0.0])            # (K + 1) u (|h2| |W3| + |b3|)
    np.testing.assert_allclose(zb[0], acc(3.03125) + [0.0, 2.0 ** -6, 0.0], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(zb[1], acc(3.0), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(msens, [marg(3.03125) - marg(3.015625), 0.0], rtol=1e-9, atol=1e-15)
    assert not changed.any()
    thr = 0.5 * (marg(3.03125) + marg(3.015625))                  # between the two margins
    assert mlp.flip_sensitivity(theta, X, thr)[5].tolist() == [True, False]


def test_in_step_flag_rule_counts_a_hidden_value_on_a_rounding_midpoint():
    """The oracle's in-step learned decision counts the values that an FP32 path might round
    the other way (lc_near) and flags the vehicle only when rounding one of them the other
    way could move its decision.  One candidate at v = 11.40625 m/s (input 0 = v / 20 =
    0.5703125 = 73/128, a BF16 value) and networks whose first hidden unit reads only that
    input, with weight w, feeding one unit of layer 2 with weight w2 and the left logit:
      w = 4, w2 = 1: 2.28125 and 2.28125, BF16 values: nothing counted beyond the inputs;
      w = 5: 2.8515625, halfway between 2.84375 (even, taken) and 2.859375: one more;
      w = 7: 3.9921875, halfway between 3.984375 and 4 (even, taken; the step below a power
             of two is half the step above): one more;
      w = 4, w2 = 7: layer 2 gets 15.96875, halfway between 15.9375 and 16 (taken): one more.
    The inputs near a boundary are counted as the reading states them (within
    2^-22 |f| + the absolute part of each input's bound).  Every margin is far from the
    threshold and each value rounded the other way moves it little, so nothing is flagged."""
    import math as _m
    import netkit
    net = synth.grid_network(2, 2, 2, 300.0, 30, 3, "zero")
    e = int(np.nonzero((net.edge_from == 0) & (net.edge_to == 1))[0][0])
    l0 = int(net.edge_lane0[e])
    nxt = int(net.succ_edge[net.succ_off[l0]])
    v = 11.40625
    se = (P["idm_s0"] + v * P["idm_T"]) / _m.sqrt(1 - (v / 13.9) ** 4)
    dem = netkit.vehicles([l0, l0], [100.0, 100.0 + P["veh_len"] + se], [v, v], [[e, nxt]] * 2)
    in_abs = np.zeros(16)
    in_abs[[2, 6, 8, 13, 15]] = 1e-5
    in_abs[[4, 10, 11]] = 5e-5
    near = {}
    cases = [(4.0, 1.0), (5.0, 1.0), (7.0, 1.0), (4.0, 7.0)]
    for w, w2 in cases:
        p = {k: np.zeros(sh) for k, sh in mlp.SHAPES}
        p["W1"][0, 0] = w
        p["W2"][0, 0] = w2
        p["W3"][1, 0] = 1.0
        o = oracle.Oracle(net, dem, P)
        o.set_lc_model(mlp.pack(p).astype(np.float32), 0.2)
        _, d = o.step(debug=True)
        assert d["lc_learn"][0] == 1 and d["lc_dir"][0] == 1 and d["flag"][0] == 0, (w, w2)
        f = d["lc_feat"][0]
        assert f[0] == v / 20.0
        n_in = int(mlp._near_alt(f, mlp.bf16(f), 2.0 ** -22 * np.abs(f) + in_abs)[0].sum())
        near[(w, w2)] = int(d["lc_near"][0]) - n_in
    assert near == {(4.0, 1.0): 0, (5.0, 1.0): 1, (7.0, 1.0): 1, (4.0, 7.0): 1}, near
    # a tie that rounds up, with the BF16 value below as the other side: at v = 10.078125
    # input 0 is 0.50390625 and weight 6 gives 3.0234375, halfway between 3.015625 and the
    # even 3.03125 (taken); weight 4 gives 2.015625, a BF16 value
    v = 10.078125
    se = (P["idm_s0"] + v * P["idm_T"]) / _m.sqrt(1 - (v / 13.9) ** 4)
    dem = netkit.vehicles([l0, l0], [100.0, 100.0 + P["veh_len"] + se], [v, v], [[e, nxt]] * 2)
    near = {}
    for w in (6.0, 4.0):
        p = {k: np.zeros(sh) for k, sh in mlp.SHAPES}
        p["W1"][0, 0] = w
        p["W2"][0, 0] = 1.0
        p["W3"][1, 0] = 1.0
        o = oracle.Oracle(net, dem, P)
        o.set_lc_model(mlp.pack(p).astype(np.float32), 0.2)
        _, d = o.step(debug=True)
        assert d["lc_learn"][0] == 1 and d["lc_dir"][0] == 1 and d["flag"][0] == 0, w
        f = d["lc_feat"][0]
        n_in = int(mlp._near_alt(f, mlp.bf16(f), 2.0 ** -22 * np.abs(f) + in_abs)[0].sum())
        near[w] = int(d["lc_near"][0]) - n_in
    assert near == {6.0: 1, 4.0: 0}, near


@pytest.mark.parametrize("t0", [0, 1])
def test_tied_classes_go_to_the_lower_index(t0):
    """A network whose left and right logits tie (0, 0) above stay (-8), decided with a
    fallback threshold of 0 (the margin of a tie is 0): the class is the lower index, left,
    so every learned candidate moves left on a step that allows it and stays on one that
    allows only moves to the right."""
    p = {k: np.zeros(s) for k, s in mlp.SHAPES}
    p["b3"][0] = -8.0
    theta = mlp.pack(p).astype(np.float32)
    net, dem = _workload()
    st, dr, dl = _pair(net, dem, t0, theta, margin=0.0)
    L = dl["lc_learn"] == 1
    assert L.sum() > 50
    assert np.all(dl["lc_margin"][L] == 0.0)
    assert np.all(dl["lc_dir"][L] == (1 if t0 % 2 == 0 else 0))


def test_mandatory_changes_bypass_the_network():
    """A vehicle on a 3-lane approach's right-turn-only lane whose route goes straight must
    move left: that change is mandatory, so an always-stay network does not decide it (no
    learned record) and the vehicle moves left as under the rule."""
    import netkit
    p = {k: np.zeros(s) for k, s in mlp.SHAPES}
    p["b3"][0] = 8.0
    theta = mlp.pack(p).astype(np.float32)
    net = synth.grid_network(3, 3, 3, 300.0, green=30, yellow=3)
    e = [k for k in range(net.n_edges) if net.edge_from[k] == 3 and net.edge_to[k] == 4][0]
    ex = [k for k in range(net.n_edges) if net.edge_from[k] == 4 and net.edge_to[k] == 5][0]
    l0 = int(net.edge_lane0[e])
    dem = netkit.vehicles([l0], [150.0], [13.9], [[e, ex]])
    o = oracle.Oracle(net, dem, P)
    o.set_lc_model(theta, 0.2)
    _, d = o.step(debug=True)
    assert d["lc_cand"][0] == 1 and d["lc_learn"][0] == 0 and d["lc_dir"][0] == 1



def _tie_net(w, w2, b1=0.0, b3=0.0):
    p = {k: np.zeros(s) for k, s in mlp.SHAPES}
    p["W1"][0, 0] = w
    p["W2"][0, 0] = w2
    p["W3"][1, 0] = 1.0
    p["b1"][0] = b1
    p["b3"][1] = b3
    return mlp.pack(p)


@pytest.mark.parametrize("x0, w, w2, alt_logit", [
    (73 / 128, 4.0, 1.0, None),            # 2.28125 and 2.28125: BF16 values, nothing near
    (73 / 128, 5.0, 1.0, 2.859375),        # 2.8515625 -> 2.84375 (even, below); other side above
    (73 / 128, 7.0, 1.0, 3.984375),        # 3.9921875 -> 4 (even); other side 4 - 2^-6 (half step)
    (129 / 256, 6.0, 1.0, 3.015625),       # 3.0234375 -> 3.03125 (even, above); other side below
    (73 / 128, 4.0, 7.0, 15.9375),         # layer 2: 15.96875 -> 16 (even); other side 16 - 2^-4
])
def test_flag_rule_in_every_rounding_position(x0, w, w2, alt_logit):
    """forward_bf16's near flag and flip_sensitivity's re-evaluation on ties in each position
    the BF16 rounding can leave one: a hidden value exactly halfway between two BF16 values
    below or above the even one taken, just under a power of two (where the step below is half
    the step above), in hidden layer 1 or 2.  The logit then moves to the value computed by
    hand for the other side, the logit bound gains that move on top of the accumulation bound
    (K + 1) 2^-22 (|h2| |W3| + |b3|), the margin bound gains the softmax difference, and the
    decision changes only when the threshold lies between the two margins.  The left logit
    carries a bias of 1/4."""
    b3 = 0.25
    theta = _tie_net(w, w2, b3=b3)
    X = np.zeros((1, 16))
    X[0, 0] = x0
    u = 2.0 ** -22
    z, near, zb_f = mlp.forward_bf16(theta, X)
    l1 = z[0, 1]
    acc = 65 * u * l1                      # |h2| |W3| + |b3| = (l1 - b3) + b3
    alt_logit = None if alt_logit is None else alt_logit + b3
    np.testing.assert_allclose(zb_f[0], [0.0, acc, 0.0], rtol=1e-12, atol=1e-18)
    assert bool(near[0]) == (alt_logit is not None)
    marg = lambda v: (np.exp(v) - 1.0) / (np.exp(v) + 2.0)
    z2, m, c, zb, msens, changed = mlp.flip_sensitivity(theta, X, 0.2)
    np.testing.assert_array_equal(z2, z)
    assert c[0] == 1 and not changed[0]
    if alt_logit is None:
        np.testing.assert_allclose(zb[0], [0.0, acc, 0.0], rtol=1e-12, atol=1e-18)
        assert msens[0] == 0.0
        return
    np.testing.assert_allclose(zb[0], [0.0, acc + abs(alt_logit - l1), 0.0], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(msens[0], abs(marg(alt_logit) - marg(l1)), rtol=1e-6, atol=1e-15)
    thr = 0.5 * (marg(alt_logit) + marg(l1))
    assert mlp.flip_sensitivity(theta, X, thr)[5][0]


def test_flag_rule_on_an_input_tie_and_the_prediction_margin():
    """An input given in FP64 exactly halfway between two BF16 values (1 + 2^-8: 1 is taken)
    is flagged when the caller passes the inputs' bound, and rounding it the other way moves
    the logit by 2^-7 through a network that passes it on with a bias of 1/4 in hidden layer
    1 and in the logit; mlp.predict's margin is the top softmax probability minus the
    second."""
    theta = _tie_net(1.0, 1.0, b1=0.25, b3=0.25)                      # 1 + 1/4 + 1/4
    X = np.zeros((1, 16))
    X[0, 0] = 1.0 + 2.0 ** -8
    z, m, c, zb, msens, changed = mlp.flip_sensitivity(theta, X, 0.2, in_delta=np.full((1, 16), 1e-9))
    assert z[0, 1] == 1.5
    acc = 65 * 2.0 ** -22 * (1.25 + 0.25)
    np.testing.assert_allclose(zb[0, 1], acc + 2.0 ** -7, rtol=1e-12)
    _, _, _, zb0, _, _ = mlp.flip_sensitivity(theta, X, 0.2)          # inputs taken as BF16
    np.testing.assert_allclose(zb0[0, 1], acc, rtol=1e-12)
    cls, mg = mlp.predict(theta, X)
    p = np.exp([0.0, 1.0 + 2.0 ** -8 + 0.5, 0.0])
    p /= p.sum()
    assert cls[0] == 1 and mg[0] == pytest.approx(p[1] - p[0], rel=1e-12)


def test_flag_rule_forward_matches_the_bf16_forward_with_biases():
    """flip_sensitivity evaluates the same BF16 network as forward_bf16 (pinned above): equal
    logits on random inputs through a random network with biases."""
    rng = np.random.default_rng(9)
    theta = mlp.init(2) + rng.normal(scale=0.1, size=mlp.N_PARAMS)
    X = rng.normal(size=(200, 16))
    z, _, _ = mlp.forward_bf16(theta, X)
    np.testing.assert_array_equal(mlp.flip_sensitivity(theta, X, 0.2)[0], z)
