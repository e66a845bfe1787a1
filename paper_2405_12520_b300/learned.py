"""Learned lane-change surrogate: data collection, GPU training and evaluation.

The network (16 -> 64 -> 64 -> 3, ReLU, softmax over stay / left / right) is trained on
(features, decision) pairs logged by the rule-based step (randomized MOBIL) and then
replaces the rule's incentive decision in the step kernel, falling back to the rule when
its softmax margin is low.  The paper's lane-change model is rule-based (Sec. III-A);
this surrogate is the library's addition.  Every numerical step (logging, forward,
backward, Adam, inference) runs in libmoss103's CUDA kernels; torch only holds device
buffers and draws minibatch indices.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import moss, synth


def collect(workloads, params, steps: int, cap: int, device="cuda"):
    """Run each (net, dem) for `steps` rule-based steps, logging candidates; returns
    (x bf16 [n,16], y int32 [n]) device tensors."""
    import torch
    x = torch.empty((cap, 16), dtype=torch.bfloat16, device=device)
    y = torch.empty(cap, dtype=torch.int32, device=device)
    total = 0
    for net, dem in workloads:
        if total >= cap:
            break
        n = torch.zeros(1, dtype=torch.int32, device=device)
        s = moss.Sim(params)
        s.load_network(net)
        s.add_vehicles(dem)
        s.set_lc_log(x[total:], y[total:], n)
        s.step(steps)
        s.sync()
        total += min(int(n.item()), cap - total)
        s.destroy()
    return x[:total], y[:total]


def class_weights(y, power: float = 0.25):
    """Inverse-frequency class weights (softened by `power`), normalised to mean 1."""
    import torch
    cnt = torch.bincount(y.long(), minlength=3).double().cpu().numpy()
    w = (cnt.sum() / np.maximum(cnt, 1.0)) ** power
    return (w / w.mean()).astype(np.float32), cnt


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases (same layout as the C ABI)."""
    rng = np.random.default_rng(seed)
    parts = []
    for shp in ((64, 16), (64,), (64, 64), (64,), (3, 64), (3,)):
        if len(shp) == 2:
            lim = math.sqrt(6.0 / shp[1])
            parts.append(rng.uniform(-lim, lim, size=shp).ravel())
        else:
            parts.append(np.zeros(shp))
    return np.concatenate(parts).astype(np.float32)


def train(x, y, epochs: int = 3, batch: int = 8192, lr: float = 1e-3, seed: int = 0, class_w=None,
          theta0=None, log_every: int = 0):
    """Adam on class-weighted cross-entropy with the library's GPU kernels; returns the
    parameters (numpy float32) and a training log."""
    import torch
    dev = x.device
    theta = torch.tensor(init_params(seed) if theta0 is None else theta0, device=dev)
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    work = torch.zeros(moss.MLP_WORK_FLOATS, dtype=torch.float32, device=dev)
    if class_w is None:
        class_w, _ = class_weights(y)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    n = x.shape[0]
    t = 0
    log = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g, device=dev).to(torch.int32)
        for b0 in range(0, n, batch):
            t += 1
            want = log_every and t % log_every == 0
            loss = moss.mlp_train_step(x, y, perm[b0:b0 + batch], theta, m, v, t, lr, class_w, work, want_loss=want)
            if want:
                log.append((t, loss))
    torch.cuda.synchronize()
    return theta.cpu().numpy(), dict(steps=t, seconds=time.perf_counter() - t0, log=log,
                                     class_w=list(map(float, class_w)))


def evaluate(theta, x, y, margin: float = 0.2):
    """Decision agreement of the network with the rule on logged samples: overall, per
    class, and with the low-margin rule fallback."""
    import torch
    dev = x.device
    th = torch.tensor(theta, device=dev)
    work = torch.zeros(moss.MLP_WORK_FLOATS, dtype=torch.float32, device=dev)
    cls = torch.empty(x.shape[0], dtype=torch.int32, device=dev)
    mar = torch.empty(x.shape[0], dtype=torch.float32, device=dev)
    moss.mlp_predict(x, th, work, cls, mar)
    yy = y.long()
    pred = cls.long()
    fb = mar < margin
    final = torch.where(fb, yy, pred)
    out = dict(n=int(x.shape[0]), agree_net=float((pred == yy).double().mean()),
               agree_with_fallback=float((final == yy).double().mean()), fallback=float(fb.double().mean()))
    for c, name in enumerate(("stay", "left", "right")):
        m = yy == c
        out[f"n_{name}"] = int(m.sum())
        out[f"agree_{name}"] = float((final[m] == c).double().mean()) if int(m.sum()) else float("nan")
    return out


def small_grid_runs(n_seeds: int, first_seed: int = 100):
    """The small plain-method workload (4x4 grid, 500 trips) under different seeds."""
    return [synth.small_grid_workload(s) for s in range(first_seed, first_seed + n_seeds)]
