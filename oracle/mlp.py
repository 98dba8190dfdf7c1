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

simulate_scheme is the full Euler scheme (Eq. (log-LIB-SDE-2), drift of
Eq. (LIBOR-drift-PT)) whose jump compensator is the network's,
A_i = C_i + s_y f(x_i), in FP64 on the oracle's own Philox increments; it is
the definition the GPU's LLL_MLP kernels are compared with path by path.
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


def forward_vec(params, x):
    """All output columns [rows, outputs] (vector head)."""
    h = x
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        h = silu(z) if li + 1 < len(params) else z
    return h


def _backprop(params, acts, zs, d):
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        grads[li] = (d.T @ acts[li], d.sum(axis=0))
        if li > 0:
            d = (d @ W) * silu_grad(zs[li - 1])
    return grads


def loss_and_grads_vec(params, x, y, n):
    """Vector head: MSE over the first n output columns (the rates; the rest
    is padding) and its gradients."""
    _, (acts, zs) = forward(params, x)
    out = zs[-1]
    r = out[:, :n] - y[:, :n]
    loss = float(np.mean(r * r))
    d = np.zeros_like(out)
    d[:, :n] = (2.0 / r.size) * r
    return loss, _backprop(params, acts, zs, d)


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


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as FP32: the
    representation in which the GPU stores the network's weights."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def params_from_flat(flat, offsets, layers, hidden, in_dim, in_pad, outputs=1):
    """The network held by the GPU as FP64 (W, b) pairs: hidden-layer and
    output weights as their BF16 values, biases FP32.  ``offsets`` are the
    flat offsets W_0, b_0, ..., W_{L-1}, b_{L-1}, w_out, b_out; the output
    layer has ``outputs`` rows (1, or n padded for the vector head)."""
    flat = np.asarray(flat, dtype=np.float32)
    params = []
    for l in range(layers):
        din = in_pad if l == 0 else hidden
        W = bf16_round(flat[offsets[2 * l]: offsets[2 * l] + hidden * din]).reshape(hidden, din)
        W = W[:, :in_dim] if l == 0 else W
        b = flat[offsets[2 * l + 1]: offsets[2 * l + 1] + hidden]
        params.append((W.astype(np.float64), b.astype(np.float64)))
    wout = bf16_round(flat[offsets[2 * layers]: offsets[2 * layers] + outputs * hidden]).astype(np.float64)
    params.append((wout.reshape(outputs, hidden),
                   flat[offsets[2 * layers + 1]: offsets[2 * layers + 1] + outputs].astype(np.float64)))
    return params


def simulate_scheme(model, params, scales, path0=0, npaths=None, strikes=None, head=0):
    """Full Euler scheme with the learned compensator, FP64, paths
    path0 .. path0 + npaths - 1 of the model's Philox streams.

    Per step k (left point t_k) and live rate i (k < i s):
      x_i = (t_k s_t, i s_i, lambda(t_k, T_i) s_lam, u_0, u_1, .., u_n),
      u_m = (log L_m(t_k) - log L_m(0)) s_u (u_0 = 0, the spot rate is fixed),
      A_i = C_i(t_k) + s_y f(x_i),  C_i = int (e^{lambda_i x} - 1 - lambda_i x) F(dx)
            (the compensator with every later weight zero, from the oracle's rule),
      log L_i(t_{k+1}) = log L_i(t_k) - A_i h + lambda_i dH_k,
    all rates of a step using the state at t_k.  Vector head (head = 1): one
    row per path, x = (t_k s_t, u_0, .., u_n), and A_i = C_i + s_y f(x)_{i-1}.
    Caplet payoffs at each T_m as in Eq. (caplet).  Returns
    snap[p, m-1, l-1] = log L_l(T_m) (l >= m) and the payoff sums and prices."""
    from . import analytic
    from . import oracle as ora

    wl = model.wl
    n, s = wl.N - 1, wl.s
    S, h = n * s, wl.delta / s
    npaths = wl.paths if npaths is None else int(npaths)
    strikes = np.asarray(wl.strikes if strikes is None else strikes, dtype=np.float64)
    ns = strikes.shape[1]
    s_t, s_i, s_lam, s_u, s_y = (float(v) for v in scales)
    dH, _ = ora.increments(model, path0, npaths)
    lam = np.asarray(wl.lam, dtype=np.float64).reshape(S, n)
    # C_i(t_k): the compensator with every later weight zero, i.e. the rule's
    # jump cumulant at lambda(t_k, T_i) (entries of rates already fixed,
    # t_k >= T_i, are never used and may overflow)
    with np.errstate(over="ignore", invalid="ignore"):
        C = analytic.kappa_quad(lam.reshape(-1), model.x, model.W).reshape(S, n)
    logL0 = np.log(np.asarray(wl.L0, dtype=np.float64)[1:])
    U = np.zeros((npaths, n))
    snap = np.full((npaths, n, n), np.nan)
    s1 = np.zeros((n, ns))
    s2 = np.zeros((n, ns))
    BN = ora.discount_terminal(wl)
    for k in range(S):
        imin = k // s + 1
        live = np.arange(imin, n + 1)
        if head:
            X = np.zeros((npaths, 1 + wl.N))
            X[:, 0] = k * h * s_t
            X[:, 2:] = U * s_u
            f = forward_vec(params, X)[:, live - 1]
        else:
            X = np.zeros((npaths, len(live), 3 + wl.N))
            X[:, :, 0] = k * h * s_t
            X[:, :, 1] = live * s_i
            X[:, :, 2] = lam[k, live - 1] * s_lam
            X[:, :, 4:] = U[:, None, :] * s_u
            f, _ = forward(params, X.reshape(-1, X.shape[-1]))
            f = f.reshape(npaths, len(live))
        A = C[k, live - 1][None, :] + s_y * f
        U[:, live - 1] += -A * h + lam[k, live - 1][None, :] * dH[:, k:k + 1]
        if (k + 1) % s == 0:
            m = imin
            logL = logL0 + U
            snap[:, m - 1, m - 1:] = logL[:, m - 1:]
            num = np.prod(1.0 + wl.delta * np.exp(logL[:, m:]), axis=1)
            Lm = np.exp(logL[:, m - 1])
            for q in range(ns):
                pay = wl.delta * BN * num * np.maximum(Lm - strikes[m - 1, q], 0.0)
                s1[m - 1, q] = pay.sum()
                s2[m - 1, q] = (pay * pay).sum()
    return dict(snap=snap, sum=s1, sumsq=s2, npaths=npaths, **ora.moments(s1, s2, npaths))


def adam_state(params):
    return [((np.zeros_like(W), np.zeros_like(W)), (np.zeros_like(b), np.zeros_like(b)))
            for W, b in params]
