"""FP64 CPU reference of the learned lane-change surrogate -- TEST INFRASTRUCTURE.

The network is the learned replacement of the MOBIL incentive decision (the paper's
lane-change model is rule-based, Sec. III-A; the surrogate is this library's addition):
16 features -> Linear(64) + ReLU -> Linear(64) + ReLU -> Linear(3) -> softmax over
{stay, left, right}, trained with class-weighted cross-entropy and Adam.  Only tests/,
__graft_entry__.smoke() and bench.py may import this module.  Plain numpy in float64; no
blocking or fusion beyond the layer definitions.

Parameter layout (one flat vector, float): W1[64,16], b1[64], W2[64,64], b2[64], W3[3,64],
b3[3] -- row-major, out x in.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 16, 64, 3
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def init(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / shp[1])
            p[name] = rng.uniform(-lim, lim, size=shp)
        else:
            p[name] = np.zeros(shp)
    return pack(p)


def forward(theta, X):
    """Logits and the activations of every layer."""
    p = unpack(theta)
    X = np.asarray(X, np.float64)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["W3"].T + p["b3"]
    return z, (X, a1, h1, a2, h2)


def softmax(z):
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def loss(theta, X, y, w_class):
    """Class-weighted mean cross-entropy: sum_i w[y_i] * -log p_i[y_i] / sum_i w[y_i]."""
    z, _ = forward(theta, X)
    p = softmax(z)
    w = np.asarray(w_class, np.float64)[y]
    return float(np.sum(w * -np.log(p[np.arange(len(y)), y])) / np.sum(w))


def grad(theta, X, y, w_class):
    """Analytic gradient of loss() by the chain rule, layer by layer."""
    prm = unpack(theta)
    z, (X, a1, h1, a2, h2) = forward(theta, X)
    p = softmax(z)
    w = np.asarray(w_class, np.float64)[y]
    W = np.sum(w)
    dz = p.copy()
    dz[np.arange(len(y)), y] -= 1.0
    dz *= (w / W)[:, None]
    g = {"W3": dz.T @ h2, "b3": dz.sum(0)}
    dh2 = dz @ prm["W3"]
    da2 = dh2 * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    dh1 = da2 @ prm["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(0)
    return pack(g)


def adam_step(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; t counts from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def predict(theta, X, margin=0.0):
    """Class and softmax margin (top1 - top2) per sample."""
    p = softmax(forward(theta, X)[0])
    s = np.sort(p, axis=1)
    return p.argmax(1), s[:, -1] - s[:, -2]


def bf16(a):
    """Nearest BF16 value (8 significant bits, ties to even) of every element, as float64."""
    a = np.asarray(a, np.float64)
    m, e = np.frexp(a)
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


def forward_bf16(theta, X):
    """The network as it runs in BF16 with FP32 accumulation: the inputs, the weights and
    both hidden layers (after bias and ReLU) rounded to BF16; biases as given; sums in
    float64.  Returns the logits; per sample, whether a hidden value lies within an FP32
    path's accumulation error of a BF16 rounding boundary, (K + 1) 2^-22 (sum of |terms| +
    |bias|), K the fan-in (there the FP32 path may round the other way); and per logit the
    same bound on the FP32 sum of the last layer (the logit tolerance where no hidden value
    is near a boundary)."""
    p = unpack(theta)
    W1, W2, W3 = bf16(p["W1"]), bf16(p["W2"]), bf16(p["W3"])
    Xb = bf16(X)
    u = 2.0 ** -22
    near = np.zeros(Xb.shape[0], bool)

    def layer(h, W, b):
        nonlocal near
        a = h @ W.T + b
        mag = np.abs(h) @ np.abs(W).T + np.abs(b)
        hv = np.maximum(a, 0.0)
        r = bf16(hv)
        # distance of hv to the midpoints between r and its BF16 neighbours
        _, e = np.frexp(np.where(r > 0, r, 1.0))
        ulp = np.ldexp(1.0, e - 8)
        ulp_in = np.where(r == np.ldexp(1.0, e - 1), ulp / 2, ulp)
        d = np.minimum(np.abs(hv - (r + ulp / 2)), np.abs(hv - (r - ulp_in / 2)))
        near |= np.any((r > 0) & (d <= (W.shape[1] + 1) * u * mag), axis=1)
        return r
    h1 = layer(Xb, W1, p["b1"])
    h2 = layer(h1, W2, p["b2"])
    zb = (W3.shape[1] + 1) * u * (np.abs(h2) @ np.abs(W3).T + np.abs(p["b3"]))
    return h2 @ W3.T + p["b3"], near, zb


def margin_class(z):
    """Softmax margin (top1 - top2) and argmax class (lowest index on ties) per row."""
    p = softmax(z)
    s = np.sort(p, axis=1)
    return s[:, -1] - s[:, -2], p.argmax(1)


def _near_alt(v, r, delta):
    """Values v (rounded to BF16 as r) within delta of a BF16 rounding boundary, and the
    value the other side of that boundary rounds to."""
    a = np.abs(r)
    _, e = np.frexp(np.where(a > 0, a, 1.0))
    ulp = np.ldexp(1.0, e - 8)
    ulp_in = np.where(a == np.ldexp(1.0, e - 1), ulp / 2, ulp)
    up, dn = a + ulp, a - ulp_in
    av = np.abs(v)
    n_up = (a > 0) & (np.abs(av - (a + up) / 2) <= delta)
    n_dn = (a > 0) & ~n_up & (np.abs(av - (a + dn) / 2) <= delta)
    alt = np.sign(r) * np.where(n_up, up, dn)
    return n_up | n_dn, alt


def flip_sensitivity(theta, X, thr, in_delta=None, chunk=65536):
    """The BF16 network of forward_bf16 with, per sample, the effect of every value that
    an FP32 path might round the other way (reading R19's flag rule): each hidden value
    within (K + 1) 2^-22 (sum of |terms| + |bias|) of a BF16 rounding boundary, and each
    input within in_delta of one (in_delta [n, 16] or None: the inputs are given in BF16),
    is rounded the other way alone and the network re-evaluated.  Returns the logits z,
    margin m, class c, a logit bound (last-layer accumulation bound plus the summed logit
    changes), the summed margin changes, and whether any such change alters the decision
    (class, or fallback when m < thr)."""
    p = unpack(theta)
    W1, W2, W3 = bf16(p["W1"]), bf16(p["W2"]), bf16(p["W3"])
    b1, b2, b3 = p["b1"], p["b2"], p["b3"]
    X = np.asarray(X, np.float64)
    Xb = bf16(X)
    u = 2.0 ** -22

    def decision(c, m):
        return np.where(m < thr, -1, c)

    def tail(h1):   # layers 2 and 3 from BF16 hidden layer 1
        a2 = h1 @ W2.T + b2
        return a2, bf16(np.maximum(a2, 0.0))

    a1 = Xb @ W1.T + b1
    h1 = bf16(np.maximum(a1, 0.0))
    n1, alt1 = _near_alt(np.maximum(a1, 0.0), h1, 17 * u * (np.abs(Xb) @ np.abs(W1).T + np.abs(b1)))
    a2, h2 = tail(h1)
    n2, alt2 = _near_alt(np.maximum(a2, 0.0), h2, 65 * u * (np.abs(h1) @ np.abs(W2).T + np.abs(b2)))
    z = h2 @ W3.T + b3
    zb = 65 * u * (np.abs(h2) @ np.abs(W3).T + np.abs(b3))
    m, c = margin_class(z)
    dec = decision(c, m)
    n = X.shape[0]
    msens = np.zeros(n)
    changed = np.zeros(n, bool)

    def account(s, z2):
        m2, c2 = margin_class(z2)
        np.add.at(msens, s, np.abs(m2 - m[s]))
        np.add.at(zb, s, np.abs(z2 - z[s]))
        changed[s[decision(c2, m2) != dec[s]]] = True

    s, j = np.nonzero(n2)                     # hidden layer 2: the logits change linearly
    for o in range(0, s.size, chunk):
        ss, jj = s[o:o + chunk], j[o:o + chunk]
        account(ss, z[ss] + (alt2[ss, jj] - h2[ss, jj])[:, None] * W3[:, jj].T)
    s, j = np.nonzero(n1)                     # hidden layer 1: layer 2 rounds again
    for o in range(0, s.size, chunk):
        ss, jj = s[o:o + chunk], j[o:o + chunk]
        a2p = a2[ss] + (alt1[ss, jj] - h1[ss, jj])[:, None] * W2[:, jj].T
        account(ss, bf16(np.maximum(a2p, 0.0)) @ W3.T + b3)
    if in_delta is not None:                  # inputs: the whole network again
        ni, alti = _near_alt(X, Xb, in_delta)
        s, k = np.nonzero(ni)
        for o in range(0, s.size, chunk):
            ss, kk = s[o:o + chunk], k[o:o + chunk]
            xa = Xb[ss].copy()
            xa[np.arange(ss.size), kk] = alti[ss, kk]
            _, h2a = tail(bf16(np.maximum(xa @ W1.T + b1, 0.0)))
            account(ss, h2a @ W3.T + b3)
    return z, m, c, zb, msens, changed


def grad_bf16(theta, X, y, w_class):
    """loss()'s gradient as a BF16 network with FP32 accumulation computes it: the forward of
    forward_bf16; the output gradient w[y] (p - onehot(y)) rounded to BF16 where it enters a
    product, and the hidden-layer gradients (after the ReLU mask of the BF16 activations)
    rounded to BF16; weight gradients as products of those BF16 operands, the output bias
    gradient from the unrounded output gradient, the hidden bias gradients as column sums of
    the BF16 hidden gradients; everything divided by sum w[y].  Sums in float64."""
    prm = unpack(theta)
    W1, W2, W3 = bf16(prm["W1"]), bf16(prm["W2"]), bf16(prm["W3"])
    Xb = bf16(X)
    h1 = bf16(np.maximum(Xb @ W1.T + prm["b1"], 0.0))
    h2 = bf16(np.maximum(h1 @ W2.T + prm["b2"], 0.0))
    z = h2 @ W3.T + prm["b3"]
    p = softmax(z)
    w = np.asarray(w_class, np.float64)[y]
    d = p.copy()
    d[np.arange(len(y)), y] -= 1.0
    d *= w[:, None]
    db = bf16(d)
    g = {"W3": db.T @ h2, "b3": d.sum(0)}
    da2 = bf16((db @ W3) * (h2 > 0))
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    da1 = bf16((da2 @ W2) * (h1 > 0))
    g["W1"] = da1.T @ Xb
    g["b1"] = da1.sum(0)
    return pack(g) / np.sum(w)
