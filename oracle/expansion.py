"""Drift-expansion schemes of Section 3 (Eq. (drifta), Eq. (drifta2)), FP64.

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the
benchmark).

The product prod_{l>i} (1 + w_l (e^{lambda_l x} - 1)) of the jump compensator
in Eq. (LIBOR-drift-PT) is expanded as in Eq. (product) and truncated after
the first (A') or second (A'') order; every term is then a combination of the
jump cumulant kappa(u) = int (e^{ux} - 1 - ux) F(dx):

  A'_i  = kappa(lam_i) + sum_{l>i} w_l [kappa(lam_i+lam_l) - kappa(lam_i) - kappa(lam_l)]
  A''_i = A'_i + sum_{i<k<l} w_k w_l [kappa(lam_i+lam_k+lam_l) - kappa(lam_i+lam_l)
          - kappa(lam_i+lam_k) - kappa(lam_k+lam_l) + kappa(lam_i) + kappa(lam_k) + kappa(lam_l)]

(the first-order bracket of Eq. (drifta2) with the signs the expansion gives;
see analytic.drift_jump_second_order for the printed ones).  w_l =
delta L_l / (1 + delta L_l) from the simulated rates at t_k: the expansions
replace the compensator of the full scheme.  Written here vectorised over
paths; the per-rate loops of analytic.py are the reference it is checked with.
"""
from __future__ import annotations

import numpy as np


def drift_terms(lam, kappa, order):
    """Per-step tables of the expansion for the rates with volatilities lam
    (m live rates): K1[i] = kappa(lam_i), K2[i, l] (l > i, else 0) and, for
    order 2, K3[i, k, l] (i < k < l, else 0)."""
    lam = np.asarray(lam, dtype=np.float64)
    m = len(lam)
    K1 = kappa(lam)
    P2 = kappa((lam[:, None] + lam[None, :]).reshape(-1)).reshape(m, m)
    K2 = np.triu(P2 - K1[:, None] - K1[None, :], 1)
    if order < 2:
        return K1, K2, None
    T3 = kappa((lam[:, None, None] + lam[None, :, None] + lam[None, None, :]).reshape(-1)).reshape(m, m, m)
    K3 = (T3 - P2[:, None, :] - P2[:, :, None] - P2[None, :, :]
          + K1[:, None, None] + K1[None, :, None] + K1[None, None, :])
    i, k, l = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    K3 = np.where((i < k) & (k < l), K3, 0.0)
    return K1, K2, K3


def drift(w, K1, K2, K3=None):
    """A' (K3 None) or A'' for all rates of all paths: w [P, m] -> A [P, m]."""
    A = K1[None, :] + w @ K2.T
    if K3 is not None:
        A = A + np.einsum("pk,pl,ikl->pi", w, w, K3)
    return A


def simulate_expansion(model, order, kappa, path0=0, npaths=None, strikes=None):
    """Full Euler scheme (Eq. (log-LIB-SDE-2)) whose jump compensator is A'
    (order 1) or A'' (order 2) computed with the cumulant ``kappa`` (a
    vectorised callable), on the oracle's Philox increments.  NIG driver
    (no continuous part).  Returns snapshots and payoff sums like
    oracle.simulate."""
    from . import oracle as ora

    wl = model.wl
    n, s = wl.N - 1, wl.s
    S, h, delta = n * s, wl.delta / s, wl.delta
    npaths = wl.paths if npaths is None else int(npaths)
    strikes = np.asarray(wl.strikes if strikes is None else strikes, dtype=np.float64)
    ns = strikes.shape[1]
    dH, _ = ora.increments(model, path0, npaths)
    lam = np.asarray(wl.lam, dtype=np.float64).reshape(S, n)
    Z = np.tile(np.log(np.asarray(wl.L0, dtype=np.float64)[1:]), (npaths, 1))
    snap = np.full((npaths, n, n), np.nan)
    s1 = np.zeros((n, ns))
    s2 = np.zeros((n, ns))
    BN = ora.discount_terminal(wl)
    for k in range(S):
        imin = k // s + 1
        live = slice(imin - 1, n)
        K1, K2, K3 = drift_terms(lam[k, live], kappa, order)
        L = np.exp(Z[:, live])
        w = delta * L / (1.0 + delta * L)
        A = drift(w, K1, K2, K3)
        Z[:, live] += -A * h + lam[k, live][None, :] * dH[:, k:k + 1]
        if (k + 1) % s == 0:
            m = imin
            snap[:, m - 1, m - 1:] = Z[:, m - 1:]
            num = np.prod(1.0 + delta * np.exp(Z[:, m:]), axis=1)
            Lm = np.exp(Z[:, m - 1])
            for q in range(ns):
                pay = delta * BN * num * np.maximum(Lm - strikes[m - 1, q], 0.0)
                s1[m - 1, q] = pay.sum()
                s2[m - 1, q] = (pay * pay).sum()
    return dict(snap=snap, sum=s1, sumsq=s2, npaths=npaths, **ora.moments(s1, s2, npaths))
