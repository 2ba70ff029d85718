"""FP64 oracle of the learned Ewald-correction surrogate (a 4-64-64-64-4 SiLU network).

TEST INFRASTRUCTURE ONLY: used by tests/ to check the CUDA forward and backward kernels.  Plain
numpy in float64, no batching tricks: forward pass layer by layer, backward pass by the chain rule
in reverse order.  Parameter packing (flat vector of 8900 values), shared by convention with the
library's weight-import call:
    W1[64][4], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[4][64], b4[4]
(W[out][in], y = W x + b).  The loss is the mean over samples and outputs of the squared error.

Features of one separation d under x,y-periodic / z-isolated BCs with box (Lx, b Lx, Lz):
u = |dx|/(Lx/2), v = |dy|/(b Lx/2), w = |dz|/F_net with F_net = 2 Lx max(1, b_max) (one scale for
the whole aspect range), beta = (b - b_min)/(b_max - b_min), each mapped to [-1, 1] by 2 t - 1.
"""
from __future__ import annotations

import numpy as np

SIZES = [(64, 4), (64, 64), (64, 64), (4, 64)]
NPARAM = sum(o * i + o for o, i in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    assert p.size == NPARAM
    out, k = [], 0
    for o, i in SIZES:
        W = p[k:k + o * i].reshape(o, i)
        k += o * i
        b = p[k:k + o]
        k += o
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in layers])


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init(seed=0):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases."""
    rng = np.random.default_rng(seed)
    layers = []
    for o, i in SIZES:
        bound = 1.0 / np.sqrt(i)
        layers.append((rng.uniform(-bound, bound, (o, i)), rng.uniform(-bound, bound, o)))
    return pack(layers)


def forward(p, x):
    """x: [n, 4] features -> y: [n, 4]."""
    a = np.asarray(x, dtype=np.float64)
    layers = unpack(p)
    for li, (W, b) in enumerate(layers):
        z = a @ W.T + b
        a = silu(z) if li < len(layers) - 1 else z
    return a


def loss_and_grad(p, x, t):
    """Mean squared error and its gradient with respect to the packed parameters."""
    layers = unpack(p)
    a = [np.asarray(x, dtype=np.float64)]
    zs = []
    for li, (W, b) in enumerate(layers):
        z = a[-1] @ W.T + b
        zs.append(z)
        a.append(silu(z) if li < len(layers) - 1 else z)
    y = a[-1]
    n = y.size
    loss = float(((y - t) ** 2).sum() / n)
    dz = 2.0 * (y - t) / n
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        grads[li] = (dz.T @ a[li], dz.sum(0))
        if li > 0:
            dz = (dz @ W) * silu_grad(zs[li - 1])
    return loss, pack(grads)


def features(d, Lx, b, b_min, b_max):
    d = np.atleast_2d(np.asarray(d, dtype=np.float64))
    F_net = 2.0 * Lx * max(1.0, b_max)
    u = np.abs(d[:, 0]) / (0.5 * Lx)
    v = np.abs(d[:, 1]) / (0.5 * b * Lx)
    w = np.abs(d[:, 2]) / F_net
    beta = np.full(d.shape[0], (b - b_min) / (b_max - b_min))
    return 2.0 * np.stack([u, v, w, beta], 1) - 1.0
