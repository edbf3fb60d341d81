"""FP64 CPU oracle of the warm-start MLP -- TEST INFRASTRUCTURE ONLY.

A per-node multilayer perceptron 16 -> 64 -> 64 -> 64 -> n_out (n_out = 2:
velocity; 3: velocity and density) with ReLU between layers (y = x W + b per layer, W stored [in][out]), mean-squared-error loss
and Adam.  Plain numpy in float64.  `bf16=True` rounds to bfloat16
(round-to-nearest-even) at the points where a BF16 tensor-core
implementation rounds its operands: the layer inputs (features and every
hidden activation after bias and ReLU), the weights, and in the backward pass
the output error and every hidden error before it multiplies a weight or an
activation.  Accumulation stays in float64 here.

Pins: finite differences of the loss (tests/test_oracle_mlp.py) and the
closed-form Adam step.
"""
from __future__ import annotations

import numpy as np

SIZES = (16, 64, 64, 64, 2)


def sizes(n_out=2):
    return SIZES[:-1] + (int(n_out),)


def bf16(x):
    """Round float64 values to the nearest bfloat16 (ties to even) via float32."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed: int, n_out: int = 2):
    """He-normal weights, zero biases, from a seeded generator."""
    rng = np.random.default_rng(seed)
    params = []
    S = sizes(n_out)
    for a, b in zip(S[:-1], S[1:]):
        params.append(rng.normal(0.0, np.sqrt(2.0 / a), size=(a, b)))
        params.append(np.zeros(b))
    return params


def pack(params):
    return np.concatenate([p.ravel() for p in params])


def unpack(vec, n_out: int = 2):
    out, o = [], 0
    S = sizes(n_out)
    for a, b in zip(S[:-1], S[1:]):
        out.append(np.asarray(vec[o:o + a * b], dtype=np.float64).reshape(a, b)); o += a * b
        out.append(np.asarray(vec[o:o + b], dtype=np.float64)); o += b
    return out


def n_params(n_out: int = 2):
    S = sizes(n_out)
    return sum(a * b + b for a, b in zip(S[:-1], S[1:]))


def forward(params, X, bf16_round=False):
    """Returns (Y, cache).  X: [n][16]."""
    r = bf16 if bf16_round else (lambda v: v)
    h = r(np.asarray(X, np.float64))
    acts = [h]
    pre = []
    L = len(SIZES) - 1
    for l in range(L):
        W, b = r(params[2 * l]), params[2 * l + 1]
        z = h @ W + b
        pre.append(z)
        if l < L - 1:
            h = r(np.maximum(z, 0.0))
            acts.append(h)
        else:
            h = z
    return h, (acts, pre)


def loss(params, X, T, bf16_round=False):
    Y, _ = forward(params, X, bf16_round)
    return float(np.mean(np.sum((Y - T) ** 2, axis=1)))


def gradients(params, X, T, bf16_round=False):
    """Gradients of loss = mean_i |Y_i - T_i|^2 with respect to every
    parameter, by backpropagation (same order as params)."""
    r = bf16 if bf16_round else (lambda v: v)
    Y, (acts, pre) = forward(params, X, bf16_round)
    n = X.shape[0]
    L = len(SIZES) - 1
    grads = [None] * (2 * L)
    d = 2.0 * (Y - T) / n
    for l in range(L - 1, -1, -1):
        d = r(d)
        grads[2 * l] = acts[l].T @ d
        grads[2 * l + 1] = d.sum(axis=0)
        if l > 0:
            d = (d @ r(params[2 * l]).T) * (pre[l - 1] > 0)
    return grads


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), t counted from 1; returns new lists."""
    out_p, out_m, out_v = [], [], []
    for p, g, mm, vv in zip(params, grads, m, v):
        mm = beta1 * mm + (1 - beta1) * g
        vv = beta2 * vv + (1 - beta2) * g * g
        mh = mm / (1 - beta1 ** t)
        vh = vv / (1 - beta2 ** t)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v
