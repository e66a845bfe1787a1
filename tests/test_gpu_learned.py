"""Learned lane-change surrogate: GPU gradients vs the FP64 reference, training on decisions
logged from the rule-based step, and the fused learned step."""
import numpy as np
import pytest

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
    """Training data from 12 small-grid seeds, held-out data from 3 others."""
    tr = learned.collect(learned.small_grid_runs(60, 100), P, 3600, 4_000_000)
    te = learned.collect(learned.small_grid_runs(3, 500), P, 3600, 1_000_000)
    return tr, te


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


def test_training_reaches_rule_agreement(logged, torch_mod):
    (xtr, ytr), (xte, yte) = logged
    cw, cnt = learned.class_weights(ytr)
    print("train samples", xtr.shape[0], "class counts", cnt)
    assert xtr.shape[0] > 100_000 and cnt[1] > 0 and cnt[2] > 0
    theta, info = learned.train(xtr, ytr, epochs=10, batch=4096, lr=2e-3, seed=1, class_w=cw)
    ev = learned.evaluate(theta, xte, yte)
    ev0 = learned.evaluate(learned.init_params(1), xte, yte)
    print("trained", ev)
    print("untrained", ev0, "train", info["steps"], "steps", round(info["seconds"], 2), "s")
    stay_only = float((yte == 0).double().mean())
    assert ev["agree_with_fallback"] >= 0.99
    assert ev["agree_net"] > ev0["agree_net"] and ev["agree_net"] >= stay_only - 1e-3
    assert ev["agree_left"] > 0.5 and ev["agree_right"] > 0.5   # the rare classes are learned
    np.save("/tmp/moss_lc_theta.npy", theta)


def test_learned_step_runs_agrees_and_keeps_invariants(logged, torch_mod):
    (xtr, ytr), _ = logged
    theta, _ = learned.train(xtr, ytr, epochs=10, batch=4096, lr=2e-3, seed=1)
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
