"""Learned lane-change surrogate on the GPU against the oracle (reading R19).

Inference: the GPU network (ms_mlp_predict, and k_learn inside the step) against the
oracle's BF16 network -- logits within the FP32 accumulation bound plus the effect of any
value near a BF16 rounding boundary; classes and the low-margin fallback bit-exact wherever
no such value can change them and the margin is not within 1e-3 (plus that effect) of the
threshold or of a tie; in the step, whole learned single steps from identical states
against the oracle's learned step.  Training: GPU gradients
against the FP64 reference (random and logged inputs), GPU Adam against the reference
Adam, training on decisions logged from the rule-based step, and what the trained network
gains over an untrained one and over the rule-only step."""
import numpy as np
import pytest

import netkit
import oracle
import parity
from oracle import mlp as ref
from paper_2405_12520_b300 import learned, moss, synth

pytestmark = pytest.mark.gpu
P = synth.default_params()


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    return torch


@pytest.fixture(scope="module")
def logged(torch_mod):
    """Training data from 60 small-grid seeds, held-out data from 3 others."""
    tr = learned.collect(learned.small_grid_runs(60, 100), P, 3600, 4_000_000)
    te = learned.collect(learned.small_grid_runs(3, 500), P, 3600, 1_000_000)
    return tr, te


@pytest.fixture(scope="module")
def trained(logged):
    (xtr, ytr), _ = logged
    cw, cnt = learned.class_weights(ytr)
    theta, info = learned.train(xtr, ytr, epochs=10, batch=4096, lr=2e-3, seed=1, class_w=cw)
    return theta, info, cw, cnt


def _predict(torch, x, theta):
    th = torch.tensor(theta, device="cuda")
    work = torch.zeros(moss.MLP_WORK_FLOATS, device="cuda")
    n = x.shape[0]
    cls = torch.empty(n, dtype=torch.int32, device="cuda")
    mar = torch.empty(n, dtype=torch.float32, device="cuda")
    zz = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    moss.mlp_predict(x, th, work, cls, mar, logits=zz)
    return cls.cpu().numpy(), mar.cpu().numpy().astype(np.float64), zz.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("which", ["trained_logged", "noisy_random"])
def test_predict_matches_oracle_network(torch_mod, logged, trained, which):
    """ms_mlp_predict against oracle/mlp.forward_bf16 sample by sample."""
    torch = torch_mod
    if which == "trained_logged":
        theta = trained[0]
        x = logged[1][0][:200_000]
    else:
        rng = np.random.default_rng(9)
        theta = (learned.init_params(4) + rng.normal(scale=0.1, size=moss.MLP_NPARAM)).astype(np.float32)
        x = torch.tensor(rng.normal(size=(50_000, 16)), dtype=torch.bfloat16, device="cuda")
    cls, mar, zg = _predict(torch, x, theta)
    # the oracle's BF16 network with, per sample, the effect of every hidden value the FP32
    # path might round the other way (reading R19's flag rule)
    z, mg, c, zbound, msens, changed = ref.flip_sensitivity(theta.astype(np.float64),
                                                            x.float().cpu().double().numpy(), 0.2)
    dz = np.abs(zg - z)
    assert np.all(dz <= zbound + 1e-6), f"logit excess {np.max(dz - zbound)}"
    assert np.all(np.abs(mar - mg) <= msens + 1e-4)
    tie = ~changed & (mg >= 1e-3 + msens)                 # no argmax tie within reach
    assert np.array_equal(cls[tie], c[tie])
    thr = ~changed & (np.abs(mg - 0.2) >= 1e-3 + msens)  # fallback decision clear
    assert np.array_equal(mar[thr] < 0.2, mg[thr] < 0.2)
    print(which, "samples", len(z), "decision sensitive to a rounding", int(changed.sum()), "max |dz|",
          float(dz.max()), "class compared", int(tie.sum()), "fallback compared", int(thr.sum()))
    assert tie.mean() > 0.95 and thr.mean() > 0.95


def _learned_case(net, dem, params, theta, margin, t0, steps=6):
    sim = parity.gpu_sim(net, dem, params)
    sim.set_lc_model(theta, margin)
    st = sim.read_state()
    st["t"] = t0
    sim.write_state(st)
    orc = oracle.Oracle(net, dem, params)
    orc.set_lc_model(theta, margin)
    rep, lrep = [], []
    for _ in range(steps):
        _, gd, gs, od, os_ = parity.step_pair(sim, orc)
        parity.compare_step(gd, gs, od, os_, dem.n, report=rep)
        parity.compare_learned(gd, od, theta, report=lrep)
    tot = {k: sum(r[k] for r in rep) for k in rep[0]}
    ltot = {k: sum(r[k] for r in lrep) for k in lrep[0] if k != "max_dz"}
    ltot["max_dz"] = max(r["max_dz"] for r in lrep)
    return tot, ltot


@pytest.mark.parametrize("net_kind,t0", [("grid12x3", 0), ("grid12x3", 31), ("delaunay", 64)])
@pytest.mark.parametrize("model", ["trained", "untrained"])
def test_learned_single_steps_match_oracle(torch_mod, trained, net_kind, t0, model):
    """The in-step learned decision (candidates listed by the decide kernel, the network in
    k_learn, margin fallback, update finished there) from identical states against the
    oracle's learned step: every vehicle's neighbours, decisions, lane, position and speed
    as in the rule step's parity, and the network's inputs and logits per candidate."""
    if net_kind == "grid12x3":
        net = synth.grid_network(12, 12, 3, 200.0, 30, 3, "wave")
        dem = synth.merge_demands(synth.place_vehicles(net, 6000, seed=70 + t0, min_spacing=7.0, internal_frac=0.3),
                                  synth.uniform_trips(net, 800, 40, seed=71 + t0))
    else:
        net = synth.delaunay_network(120, box=3000.0, seed=7)
        dem = synth.merge_demands(synth.place_vehicles(net, 2500, seed=72, min_spacing=6.0, internal_frac=0.4),
                                  synth.uniform_trips(net, 400, 40, seed=73))
    if model == "trained":
        theta, margin = trained[0], 0.2
    else:   # an untrained network with a small margin: many changes, most by the network
        theta, margin = learned.init_params(7), 0.05
    tot, ltot = _learned_case(net, dem, dict(P, seed=99 + t0), theta, margin, t0)
    print(net_kind, t0, model, tot, ltot)
    assert tot["compared"] > 0.9 * tot["active"]
    assert ltot["learned"] > 100 and ltot["exact"] > 0 and ltot["changes"] > 0
    assert ltot["learned_flagged"] <= 0.05 * (ltot["learned"] + ltot["learned_flagged"]) + 2


@pytest.mark.parametrize("variant", ["lane_limits", "max_pressure", "dynamic_lanes", "threshold_jitter"])
@pytest.mark.parametrize("model", ["trained", "untrained"])
def test_learned_single_steps_with_variants_match_oracle(torch_mod, trained, model, variant):
    """The learned step with lane speed limits on 15% of the lanes and 3% closed (R14 with
    R19: the decide and k_learn instances for lane modifications), or with max-pressure
    signals (R13 with R19), or with about 30% of the lane links closed (R17 with R19), or
    with per-trip incentive thresholds (R12: the rule's decision where the network falls
    back), against the oracle's learned step with the same setting, six steps from
    identical states."""
    net = synth.grid_network(12, 12, 3, 200.0, 30, 3, "wave")
    dem = synth.merge_demands(synth.place_vehicles(net, 6000, seed=81, min_spacing=7.0, internal_frac=0.3),
                              synth.uniform_trips(net, 800, 40, seed=82))
    rng = np.random.default_rng(83)
    lim = np.nonzero(rng.random(net.n_lanes) < 0.15)[0]
    shut = np.nonzero(rng.random(net.n_lanes) < 0.03)[0]
    vmax = rng.uniform(5.0, 12.0, lim.size).astype(np.float32)
    if model == "trained":
        theta, margin = trained[0], 0.2
    else:
        theta, margin = learned.init_params(7), 0.05
    params = dict(P, seed=141)
    if variant == "max_pressure":
        params.update(signal_mode=1, mp_interval=10)
    elif variant == "threshold_jitter":
        params.update(mobil_th_jitter=0.15)
    sim = parity.gpu_sim(net, dem, params)
    st = sim.read_state()
    st["t"] = 58 if variant == "max_pressure" else 0   # max-pressure decisions at 60 and 70
    sim.write_state(st)
    sim.set_lc_model(theta, margin)
    orc = oracle.Oracle(net, dem, params)
    orc.set_lc_model(theta, margin)
    if variant == "lane_limits":
        for side in (sim, orc):
            side.set_lane_limits(lim, vmax=vmax)
            side.set_lane_limits(shut, closed=np.ones(shut.size, np.int32))
    elif variant == "dynamic_lanes":
        mask = netkit.closable_links(net, dem, np.random.default_rng(84), 0.3)
        lanes = np.array(list(mask), np.int32)
        masks = np.array([mask[int(l)] for l in lanes], np.uint32)
        for side in (sim, orc):
            side.set_lane_links(lanes, masks)
    rep, lrep = [], []
    for _ in range(6):
        _, gd, gs, od, os_ = parity.step_pair(sim, orc)
        parity.compare_step(gd, gs, od, os_, dem.n, report=rep)
        parity.compare_learned(gd, od, theta, report=lrep)
    tot = {k: sum(r[k] for r in rep) for k in rep[0]}
    ltot = {k: sum(r[k] for r in lrep) for k in lrep[0] if k != "max_dz"}
    print(variant, model, tot, ltot)
    assert tot["compared"] > 0.9 * tot["active"]
    assert ltot["learned"] > 100 and ltot["changes"] > 0
    assert ltot["learned_flagged"] <= 0.05 * (ltot["learned"] + ltot["learned_flagged"]) + 2


def test_learned_resume_is_bit_exact(torch_mod, trained):
    """Checkpoint / resume with the learned model set: 300 + 200 steps through a state read
    back and written into a new simulation equal 500 uninterrupted steps, bit for bit."""
    net, dem = synth.small_grid_workload(4)
    theta = trained[0]
    a = parity.gpu_sim(net, dem, P, debug=False)
    a.set_lc_model(theta, 0.2)
    a.step(500)
    sa = a.read_state()
    b = parity.gpu_sim(net, dem, P, debug=False)
    b.set_lc_model(theta, 0.2)
    b.step(300)
    mid = b.read_state()
    c = parity.gpu_sim(net, dem, P, debug=False)
    c.set_lc_model(theta, 0.2)
    c.write_state(mid)
    c.step(200)
    sc = c.read_state()
    for k in ("id", "lane", "x", "v", "route_idx", "t_arr", "t"):
        np.testing.assert_array_equal(sa[k], sc[k])
    assert a.read_lc_stats()["candidates"] > 0


def test_gpu_gradient_matches_fp64_reference(torch_mod):
    torch = torch_mod
    rng = np.random.default_rng(5)
    n = 1000
    X = torch.tensor(rng.normal(size=(n, 16)), dtype=torch.bfloat16, device="cuda")
    y = torch.tensor(rng.integers(0, 3, size=n), dtype=torch.int32, device="cuda")
    idx = torch.arange(n, dtype=torch.int32, device="cuda")
    theta = learned.init_params(11) + rng.normal(scale=0.05, size=moss.MLP_NPARAM).astype(np.float32)
    cw = np.array([1.0, 3.0, 2.0], np.float32)
    g = torch.zeros(moss.MLP_NPARAM, device="cuda")
    work = torch.zeros(moss.MLP_WORK_FLOATS, device="cuda")
    moss.mlp_grad(X, y, idx, torch.tensor(theta, device="cuda"), cw, work, g)
    g_gpu = g.cpu().double().numpy()
    g_ref = ref.grad(theta.astype(np.float64), X.float().cpu().double().numpy(), y.cpu().numpy(), cw.astype(np.float64))
    cos = g_gpu @ g_ref / (np.linalg.norm(g_gpu) * np.linalg.norm(g_ref))
    rel = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    print("cosine", cos, "rel L2", rel)
    assert cos >= 0.999 and rel <= 2e-2
    # loss value of the same batch
    loss = moss.mlp_train_step(X, y, idx, torch.tensor(theta, device="cuda"), torch.zeros_like(g), torch.zeros_like(g),
                               1, 0.0, cw, work, want_loss=True)
    assert loss == pytest.approx(ref.loss(theta.astype(np.float64), X.float().cpu().double().numpy(),
                                          y.cpu().numpy(), cw), rel=2e-2)


@pytest.mark.parametrize("at", ["init", "trained"])
def test_gpu_gradient_on_logged_samples(torch_mod, logged, trained, at):
    """Gradients on the inputs the step logs (their own scales), at an initial and at the
    trained network, with the training's class weights, against the reference computed with
    the kernel's BF16 rounding points (oracle/mlp.grad_bf16) and against the plain FP64
    gradient.  At the trained network the gradient is a small residual, and the BF16
    roundings themselves move it by several per cent from the FP64 value, so the FP64
    criterion (cosine >= 0.999, relative L2 <= 2e-2) applies at the initial network only."""
    torch = torch_mod
    (xtr, ytr), _ = logged
    theta0, _, cw, _ = trained
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    idx = torch.randperm(xtr.shape[0], generator=g, device="cuda")[:4096].to(torch.int32)
    theta = learned.init_params(12) if at == "init" else theta0
    grad = torch.zeros(moss.MLP_NPARAM, device="cuda")
    work = torch.zeros(moss.MLP_WORK_FLOATS, device="cuda")
    moss.mlp_grad(xtr, ytr, idx, torch.tensor(theta, device="cuda"), cw, work, grad)
    X = xtr[idx.long()].float().cpu().double().numpy()
    Y = ytr[idx.long()].cpu().numpy()
    g_gpu = grad.cpu().double().numpy()

    def cmp(g_ref):
        cos = g_gpu @ g_ref / (np.linalg.norm(g_gpu) * np.linalg.norm(g_ref))
        return cos, np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    cos_b, rel_b = cmp(ref.grad_bf16(theta.astype(np.float64), X, Y, cw.astype(np.float64)))
    cos_f, rel_f = cmp(ref.grad(theta.astype(np.float64), X, Y, cw.astype(np.float64)))
    print(at, "vs BF16 reference: cosine", cos_b, "rel L2", rel_b, "| vs FP64: cosine", cos_f, "rel L2", rel_f)
    assert cos_b >= 0.9995 and rel_b <= 1e-2
    if at == "init":
        assert cos_f >= 0.999 and rel_f <= 2e-2


def test_gpu_adam_matches_reference_adam(torch_mod, logged):
    """Five training steps: after each, the GPU's parameters and moments equal one reference
    Adam step (oracle/mlp.adam_step, FP64) from the GPU's previous parameters and moments
    with the GPU's gradient of that minibatch, within FP32 rounding."""
    torch = torch_mod
    (xtr, ytr), _ = logged
    cw = np.array([1.0, 2.0, 2.0], np.float32)
    theta = torch.tensor(learned.init_params(21), device="cuda")
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    work = torch.zeros(moss.MLP_WORK_FLOATS, device="cuda")
    grad = torch.zeros_like(theta)
    lr = 2e-3
    for t in range(1, 6):
        idx = torch.arange((t - 1) * 4096, t * 4096, dtype=torch.int32, device="cuda")
        moss.mlp_grad(xtr, ytr, idx, theta, cw, work, grad)
        th0, m0, v0, g0 = (a.cpu().double().numpy() for a in (theta, m, v, grad))
        moss.mlp_train_step(xtr, ytr, idx, theta, m, v, t, lr, cw, work)
        th_r, m_r, v_r = ref.adam_step(th0, g0, m0, v0, t, lr=lr)
        th1, m1, v1 = (a.cpu().double().numpy() for a in (theta, m, v))
        # the gradient is summed with float atomics in both calls: order-level differences
        np.testing.assert_allclose(m1, m_r, rtol=1e-4, atol=1e-9)
        np.testing.assert_allclose(v1, v_r, rtol=1e-3, atol=1e-12)
        np.testing.assert_allclose(th1, th_r, rtol=0, atol=lr * 1e-2 + 1e-6)
        assert np.max(np.abs(th1 - th0)) > 0.5 * lr   # an update happened


def test_training_reaches_rule_agreement(logged, trained, torch_mod):
    (xtr, ytr), (xte, yte) = logged
    theta, info, cw, cnt = trained
    print("train samples", xtr.shape[0], "class counts", cnt)
    assert xtr.shape[0] > 100_000 and cnt[1] > 0 and cnt[2] > 0
    ev = learned.evaluate(theta, xte, yte)
    ev0 = learned.evaluate(learned.init_params(1), xte, yte)
    print("trained", ev)
    print("untrained", ev0, "train", info["steps"], "steps", round(info["seconds"], 2), "s")
    stay_only = float((yte == 0).double().mean())
    assert ev["agree_with_fallback"] >= 0.99
    assert ev["agree_net"] > ev0["agree_net"] and ev["agree_net"] >= stay_only - 1e-3
    assert ev["agree_left"] > 0.5 and ev["agree_right"] > 0.5   # the rare classes are learned


def test_learned_step_runs_agrees_and_keeps_invariants(trained, torch_mod):
    """A whole 3600-step small-grid run with the trained network against the rule-only run:
    decision agreement, arrivals and network mean speed per window (what the learned form
    gives up against the rule it replaces), device order/gap checks on."""
    theta = trained[0]
    net, dem = synth.small_grid_workload(777)
    rule = parity.gpu_sim(net, dem, P, debug=False, n_windows=12)
    lrn = parity.gpu_sim(net, dem, P, debug=True, n_windows=12)   # device order/gap check on
    lrn.set_lc_model(theta, 0.2)
    rule.step(3600)
    lrn.step(3600)
    lrn.sync()
    st = lrn.read_lc_stats()
    mr, ml = rule.read_metrics(), lrn.read_metrics()
    print("learned stats", st, "arrived", mr["arrived"], ml["arrived"])
    assert ml["err"] == 0
    assert st["candidates"] > 0 and st["agree"] >= 0.99 * st["candidates"]
    assert abs(ml["arrived"] - mr["arrived"]) <= 0.02 * mr["arrived"]
    # network mean speed per window within 2% of the rule run
    gv, gc = ml["vsum"].sum(1), ml["vcnt"].sum(1)
    rv, rc = mr["vsum"].sum(1), mr["vcnt"].sum(1)
    busy = rc >= 2000
    assert np.all(np.abs(gv[busy] / gc[busy] - rv[busy] / rc[busy]) <= 0.02 * rv[busy] / rc[busy])


@pytest.mark.parametrize("debug,mods", [(False, False), (True, True)])
def test_learned_path_taking_every_fallback_is_the_rule_step(torch_mod, debug, mods):
    """With margin 1 every listed candidate falls back to the rule (a near-zero network gives
    probabilities near 1/3), so the learned path (candidates listed by the decide kernel and
    finished by k_learn) must give the rule step bit for bit, with and without lane
    modifications; every candidate is counted and falls back."""
    theta = (learned.init_params(3) * 1e-3).astype(np.float32)
    net, dem = synth.small_grid_workload(778)
    rule = parity.gpu_sim(net, dem, P, debug=debug)
    lrn = parity.gpu_sim(net, dem, P, debug=debug)
    if mods:
        lanes = np.nonzero(np.asarray(net.lane_edge) >= 0)[0][::7].astype(np.int32)
        vmax = np.full(lanes.shape, 8.0, np.float32)
        for s in (rule, lrn):
            s.set_lane_limits(lanes, vmax=vmax)
    lrn.set_lc_model(theta, 1.0)
    for k in range(6):
        rule.step(50)
        lrn.step(50)
        a, b = rule.read_state(), lrn.read_state()
        for key in ("id", "lane", "x", "v", "route_idx"):
            np.testing.assert_array_equal(a[key], b[key])
    st = lrn.read_lc_stats()
    print(st)
    assert st["candidates"] > 100 and st["fallbacks"] == st["candidates"] and st["agree"] == st["candidates"]
    assert lrn.read_metrics(lanes=False)["err"] == 0
