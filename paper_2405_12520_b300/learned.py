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


def collect_batched(specs, params, steps: int, cap: int, per_batch: int = 256, device="cuda"):
    """The same logging as collect, with many small scenarios in one batched simulation
    (a disjoint union of networks stepped together): specs is a list of (seed, n_trips,
    n_placed), each the small 4x4 grid with n_trips uniform-OD trips departing over 600 s
    and n_placed vehicles already on it at t = 0, fronts 6 m apart or more (a jam; 0: none).
    Stops once cap samples are logged; returns (x bf16 [n,16], y int32 [n]) and the number
    of scenario runs used."""
    import torch
    x = torch.empty((cap, 16), dtype=torch.bfloat16, device=device)
    y = torch.empty(cap, dtype=torch.int32, device=device)
    total, runs = 0, 0
    net = synth.grid_network(4, 4, 2, 200.0, 30, 3, "zero")
    for b0 in range(0, len(specs), per_batch):
        if total >= cap:
            break
        chunk = specs[b0:b0 + per_batch]
        dems = [synth.uniform_trips(net, nt, 600, 13.9, seed=sd) if npl == 0 else
                synth.merge_demands(synth.place_vehicles(net, npl, seed=sd, min_spacing=6.0),
                                    synth.uniform_trips(net, nt, 600, 13.9, seed=sd + 1))
                for sd, nt, npl in chunk]
        n = torch.zeros(1, dtype=torch.int32, device=device)
        s = moss.Sim(params)
        s.load_network_batch([net] * len(chunk))
        s.add_vehicles_batch(dems)
        s.set_lc_log(x[total:], y[total:], n)
        s.step(steps)
        s.sync()
        total += min(int(n.item()), cap - total)
        runs += len(chunk)
        s.destroy()
    return x[:total], y[:total], runs


# (trips, vehicles placed at t = 0, share of the runs)
MIX = ((500, 0, 0.3), (1500, 0, 0.1), (3000, 0, 0.1), (5000, 0, 0.15), (500, 2500, 0.2), (300, 2900, 0.15))


def mixed_specs(n: int, first_seed: int = 10_000, mix=MIX):
    """n (seed, trips, placed) scenarios in the given shares: the small configuration's 500
    trips; denser runs whose standing queues give the network the congested cases; and runs
    that start in a jam (2,500 or 2,900 vehicles placed 6 m apart or more, then 500 or 300
    trips), without which the network meets the near-jam states of a 5M-vehicle grid too
    rarely (decision agreement there 98.5-98.8% instead of 99.5%)."""
    out, k = [], 0
    for trips, placed, share in mix:
        for _ in range(int(round(n * share))):
            out.append((first_seed + 2 * k, trips, placed))
            k += 1
    rng = np.random.default_rng(first_seed)
    order = rng.permutation(len(out))
    return [tuple(int(v) for v in out[i]) for i in order]


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
          theta0=None, log_every: int = 0, tc: bool = True):
    """Adam on class-weighted cross-entropy with the library's GPU kernels; returns the
    parameters (numpy float32) and a training log.  tc: the tcgen05 training kernel (else
    the mma.sync one)."""
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
            loss = moss.mlp_train_step(x, y, perm[b0:b0 + batch], theta, m, v, t, lr, class_w, work, want_loss=want,
                                       tc=tc)
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
