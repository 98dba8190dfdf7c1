"""FP64 multilayer perceptron (forward, backward, Adam) for the learned drift.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the
benchmark).

The learned part stands in for the jump-compensator integral of
Eq. (LIBOR-drift-PT) in the full scheme: a network f maps a row of
(t, i, lambda(t, T_i), log-rate vector) features to the state-dependent part
of the compensator, A_i - C_i, in scaled units.  This module is the plain FP64
definition of that network and of its gradients, written with numpy matrix
products; the GPU's BF16 kernels are compared with it.

Layers: x -> SiLU(x W_1^T + b_1) -> SiLU(. W_2^T + b_2) -> ... -> . w_out + b_out,
SiLU(z) = z / (1 + e^{-z}); loss = mean (f(x) - y)^2.
"""
from __future__ import annotations

import numpy as np


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(sizes, seed=0):
    """He-style uniform init, sizes = [in, h1, ..., hk, 1].  Returns list of
    (W [out, in], b [out]) in FP64."""
    rng = np.random.default_rng(seed)
    params = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / a) / np.sqrt(2.0)
        params.append((rng.uniform(-lim, lim, size=(b, a)), np.zeros(b)))
    return params


def forward(params, x):
    """Returns the output [rows] and the cache of pre-activations/activations."""
    acts = [x]
    zs = []
    h = x
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        zs.append(z)
        if li + 1 < len(params):
            h = silu(z)
            acts.append(h)
        else:
            h = z
    return h[:, 0], (acts, zs)


def loss_and_grads(params, x, y):
    """MSE loss and its gradients w.r.t. every W and b (list like params)."""
    out, (acts, zs) = forward(params, x)
    r = out - y
    loss = float(np.mean(r * r))
    d = (2.0 / len(y)) * r[:, None]  # dL/dz of the output layer
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        grads[li] = (d.T @ acts[li], d.sum(axis=0))
        if li > 0:
            d = (d @ W) * silu_grad(zs[li - 1])
    return loss, grads


def adam_step(params, grads, state, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) in place; ``state`` holds (m, v)."""
    out = []
    for (W, b), (gW, gb), st in zip(params, grads, state):
        new = []
        for p, g, (m, v) in zip((W, b), (gW, gb), st):
            m[...] = b1 * m + (1 - b1) * g
            v[...] = b2 * v + (1 - b2) * g * g
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            new.append(p - lr * mh / (np.sqrt(vh) + eps))
        out.append(tuple(new))
    return out


def adam_state(params):
    return [((np.zeros_like(W), np.zeros_like(W)), (np.zeros_like(b), np.zeros_like(b)))
            for W, b in params]
