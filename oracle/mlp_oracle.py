"""FP64 reference of the warm-start surrogate network (test infrastructure only).

A plain multilayer perceptron written from its definitions: dense layers z = x W + b,
GELU(z) = z Phi(z) with Phi the standard normal CDF (exact, erf form) on every hidden
layer, a linear output layer, the mean squared error L = mean((y - t)^2), its gradients
by the chain rule, and Adam (Kingma & Ba: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
w -= lr mhat / (sqrt(vhat) + eps)).  Only the tests and the benchmark's checks use it.

`quantize=True` rounds, to bfloat16 (round to nearest even), exactly the operands the GPU
kernels hold in bfloat16: the network input, the weights, every hidden activation fed
to the next layer, and the backward deltas fed to the weight-gradient and input-
gradient products; all arithmetic stays FP64.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def init_params(sizes, seed=0):
    """Uniform(-a, a) weights with a = sqrt(6 / (fan_in + fan_out)), zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for k, n in zip(sizes[:-1], sizes[1:]):
        a = np.sqrt(6.0 / (k + n))
        params.append([rng.uniform(-a, a, size=(k, n)), np.zeros(n)])
    return params


def forward(params, x, quantize=False):
    q = bf16 if quantize else (lambda v: v)
    acts, zs = [q(x)], []
    h = q(x)
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = h @ q(W) + b
        zs.append(z)
        if l < L - 1:
            h = q(gelu(z))
            acts.append(h)
        else:
            h = z
    return h, zs, acts


def loss_and_grads(params, x, t, quantize=False):
    """MSE loss and its gradients [(dW, db), ...] by backpropagation."""
    q = bf16 if quantize else (lambda v: v)
    y, zs, acts = forward(params, x, quantize)
    n = y.size
    loss = np.mean((y - t) ** 2)
    dz = 2.0 * (y - t) / n
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        dzq = q(dz)
        grads[l] = [acts[l].T @ dzq, dz.sum(0)]
        if l > 0:
            da = dzq @ q(W).T
            dz = da * gelu_grad(zs[l - 1])
    return loss, grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place; state = {'t': int, 'm': [...], 'v': [...]}."""
    if not state:
        state.update(t=0, m=[[np.zeros_like(W), np.zeros_like(b)] for W, b in params],
                     v=[[np.zeros_like(W), np.zeros_like(b)] for W, b in params])
    state["t"] += 1
    t = state["t"]
    for l, (p, g) in enumerate(zip(params, grads)):
        for j in range(2):
            state["m"][l][j] = b1 * state["m"][l][j] + (1 - b1) * g[j]
            state["v"][l][j] = b2 * state["v"][l][j] + (1 - b2) * g[j] ** 2
            mh = state["m"][l][j] / (1 - b1 ** t)
            vh = state["v"][l][j] / (1 - b2 ** t)
            p[j] -= lr * mh / (np.sqrt(vh) + eps)
