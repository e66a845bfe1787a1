"""The surrogate's training kernel on the 5th-generation tensor core (tcgen05 MMAs with
FP32 accumulators in tensor memory, ms_mlp_grad_tc / ms_mlp_train_step_tc) against the
oracle's BF16-emulating gradient (oracle/mlp.grad_bf16, pinned on the CPU by central
differences and closed forms), against the plain FP64 gradient at an initial network,
and against the mma.sync kernel; batches with a ragged last CTA of 128 samples."""
import numpy as np
import pytest

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
def data(torch_mod):
    """About 0.5M decisions logged by the rule step on the small grid's mixed scenarios,
    and a network trained on them (the mma.sync kernel)."""
    x, y, _ = learned.collect_batched(learned.mixed_specs(256), P, 3600, 500_000)
    cw, _ = learned.class_weights(y)
    theta, _ = learned.train(x, y, epochs=2, batch=8192, lr=2e-3, seed=1, class_w=cw, tc=False)
    return x, y, cw, theta


def _grad(torch, x, y, idx, theta, cw, tc):
    grad = torch.zeros(moss.MLP_NPARAM, device="cuda")
    work = torch.zeros(moss.MLP_WORK_FLOATS, device="cuda")
    moss.mlp_grad(x, y, idx, torch.tensor(theta, device="cuda"), cw, work, grad, tc=tc)
    torch.cuda.synchronize()
    assert work[moss.MLP_NPARAM + 2:moss.MLP_NPARAM + 3].view(torch.int32).item() == 0   # no wait ran out
    return grad.cpu().double().numpy()


def _cmp(g, g_ref):
    cos = g @ g_ref / (np.linalg.norm(g) * np.linalg.norm(g_ref))
    return cos, np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)


@pytest.mark.parametrize("at", ["init", "trained"])
@pytest.mark.parametrize("batch", [4096, 4096 + 77, 130, 1])
def test_tc_gradient_matches_bf16_reference(torch_mod, data, at, batch):
    """Per parameter block (W1, b1, W2, b2, W3, b3) and as a whole: the tcgen05 gradient
    against grad_bf16 on logged features (their own scales), and against the mma.sync
    kernel's gradient of the same minibatch (the same roundings, another summation order)."""
    torch = torch_mod
    x, y, cw, theta_tr = data
    g = torch.Generator(device="cuda")
    g.manual_seed(7 + batch)
    theta = learned.init_params(12) if at == "init" else theta_tr
    if batch == 1:
        # one sample (a CTA holding a single row): the least confident of 4,096, since for a
        # sample the network is sure of, p - 1 of the true class lies below the FP32
        # resolution of p, and that one term is then the whole gradient
        cand = torch.randperm(x.shape[0], generator=g, device="cuda")[:4096]
        z, _ = ref.forward(theta.astype(np.float64), x[cand].float().cpu().double().numpy())
        pz = np.exp(z - z.max(1, keepdims=True))
        pz /= pz.sum(1, keepdims=True)
        idx = cand[int(np.argmin(pz.max(1)))].reshape(1).to(torch.int32)
    else:
        idx = torch.randperm(x.shape[0], generator=g, device="cuda")[:batch].to(torch.int32)
    g_tc = _grad(torch, x, y, idx, theta, cw, tc=True)
    g_mma = _grad(torch, x, y, idx, theta, cw, tc=False)
    X = x[idx.long()].float().cpu().double().numpy()
    Y = y[idx.long()].cpu().numpy()
    g_b = ref.grad_bf16(theta.astype(np.float64), X, Y, cw.astype(np.float64))
    cos_b, rel_b = _cmp(g_tc, g_b)
    cos_m, rel_m = _cmp(g_tc, g_mma)
    print(at, batch, "tc vs BF16 reference: cosine", cos_b, "rel L2", rel_b, "| tc vs mma.sync rel L2", rel_m)
    assert cos_b >= 0.9995 and rel_b <= 1e-2
    assert rel_m <= 1e-3
    o = 0
    for name, shape in ref.SHAPES:
        k = int(np.prod(shape))
        o, blk = o + k, slice(o, o + k)
        if np.linalg.norm(g_b[blk]) == 0:
            continue
        _, rel = _cmp(g_tc[blk], g_b[blk])
        assert rel <= 2e-2, (name, rel)
    if at == "init" and batch >= 4096:
        cos_f, rel_f = _cmp(g_tc, ref.grad(theta.astype(np.float64), X, Y, cw.astype(np.float64)))
        assert cos_f >= 0.999 and rel_f <= 2e-2


def test_tc_gradient_on_random_inputs(torch_mod):
    """N(0, 1) features, a perturbed initial network and uneven class weights: the FP64
    criterion of the training kernels (cosine >= 0.999, relative L2 <= 2e-2) and the loss."""
    torch = torch_mod
    rng = np.random.default_rng(5)
    n = 1000
    X = torch.tensor(rng.normal(size=(n, 16)), dtype=torch.bfloat16, device="cuda")
    y = torch.tensor(rng.integers(0, 3, size=n), dtype=torch.int32, device="cuda")
    idx = torch.arange(n, dtype=torch.int32, device="cuda")
    theta = learned.init_params(11) + rng.normal(scale=0.05, size=moss.MLP_NPARAM).astype(np.float32)
    cw = np.array([1.0, 3.0, 2.0], np.float32)
    g_tc = _grad(torch, X, y, idx, theta, cw, tc=True)
    Xd, Yd = X.float().cpu().double().numpy(), y.cpu().numpy()
    cos, rel = _cmp(g_tc, ref.grad(theta.astype(np.float64), Xd, Yd, cw.astype(np.float64)))
    cos_b, rel_b = _cmp(g_tc, ref.grad_bf16(theta.astype(np.float64), Xd, Yd, cw.astype(np.float64)))
    print("random: tc vs FP64 cosine", cos, "rel", rel, "| vs BF16 reference rel", rel_b)
    assert cos >= 0.999 and rel <= 2e-2 and rel_b <= 1e-2
    work = torch.zeros(moss.MLP_WORK_FLOATS, device="cuda")
    th = torch.tensor(theta, device="cuda")
    z = torch.zeros_like(th)
    loss = moss.mlp_train_step(X, y, idx, th, z, z.clone(), 1, 0.0, cw, work, want_loss=True, tc=True)
    assert loss == pytest.approx(ref.loss(theta.astype(np.float64), Xd, Yd, cw), rel=2e-2)


def test_tc_training_follows_the_mma_kernel(torch_mod, data):
    """Twenty Adam steps from the same start with either kernel: the parameters stay within
    a small fraction of the distance they travelled."""
    torch = torch_mod
    x, y, cw, _ = data
    out = {}
    for tc in (False, True):
        theta = torch.tensor(learned.init_params(31), device="cuda")
        m = torch.zeros_like(theta)
        v = torch.zeros_like(theta)
        work = torch.zeros(moss.MLP_WORK_FLOATS, device="cuda")
        for t in range(1, 21):
            idx = torch.arange((t - 1) * 8192, t * 8192, dtype=torch.int32, device="cuda")
            moss.mlp_train_step(x, y, idx, theta, m, v, t, 2e-3, cw, work, tc=tc)
        out[tc] = theta.cpu().double().numpy()
    th0 = learned.init_params(31).astype(np.float64)
    moved = np.linalg.norm(out[False] - th0)
    diff = np.linalg.norm(out[True] - out[False])
    print("travelled", moved, "tc - mma", diff)
    assert moved > 0 and diff <= 0.05 * moved
