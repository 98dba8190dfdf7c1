"""Pins of the oracle's drift (Eq. (LIBOR-drift-PT), (Levy-LIBOR-beta)).

  * The direct product formula equals the exact drift from the product
    expansion of Eq. (product) with inclusion-exclusion over subsets, given
    the same discrete Levy measure (the rule's kappa): exact algebra, so the
    two agree to rounding.  With the closed-form (untruncated) kappa they
    agree within the tail mass beyond a.
  * The last rate's drift is -kappa(lambda_n) (the remark after
    Eq. (Levy-LIBOR-beta): L(., T_N) is a martingale).
  * The Brownian driver's drift is the log-normal LIBOR drift.
  * A - A' = O(|L|^2) (Eq. (drifta)) and A - A'' = O(|L|^3) (Eq. (drifta2)),
    the latter only with the corrected signs of the first-order bracket.
  * The frozen-curve table D0 is the running integral of the drift at L(0)
    (Eq. (Picard-2)).
"""
import math

import numpy as np
import pytest

from oracle import analytic, oracle, quadrature
from paper_1006_3340_gb300 import workloads


def _tiny(N=6, Q=16):
    wl = workloads.tiny(N=N, s=3, Q=Q)
    x, W = quadrature.rule_for(wl)
    return wl, x, W, oracle.OracleModel(wl, x, W)


@pytest.mark.parametrize("N", [3, 5, 8])
def test_direct_drift_equals_subset_expansion(N):
    wl, x, W, model = _tiny(N=N)
    n = wl.n
    rng = np.random.default_rng(N)
    kap = lambda u: float(analytic.kappa_quad(u, x, W)[0])
    for k in [0, 1, wl.steps - 1]:
        lam = wl.lam[k]
        w = rng.uniform(0.0, 0.3, size=n)
        for i in range(1, n + 1):
            b = oracle.drift(model, k, i, w)
            A = analytic.drift_jump_exact(i, w, lam, kap)
            assert abs(-b - A) < 1e-13 * max(1.0, abs(A)) + 1e-16, (k, i, b, A)


def test_direct_drift_vs_untruncated_kappa_within_tail():
    wl, x, W, model = _tiny(N=5, Q=32)
    n = wl.n
    mu = analytic.nig_mu(wl)
    kex = lambda u: float(analytic.kappa(u, wl.alpha, wl.beta, wl.dbar, mu))
    w = np.full(n, 0.02)
    lam = wl.lam[0]
    for i in range(1, n + 1):
        A = -oracle.drift(model, 0, i, w)
        Aex = analytic.drift_jump_exact(i, w, lam, kex)
        # the largest exponent in the integrand is sum(lam) <= 0.7, alpha - |beta| = 7
        tail = analytic.kappa_tail(float(lam.sum()), wl.alpha, wl.beta, wl.dbar, wl.a)
        assert abs(A - Aex) <= 2 * abs(tail) + 1e-14, (i, A, Aex, tail)


def test_last_rate_drift_is_minus_kappa():
    for wl in [workloads.small_plain(), workloads.large_single()]:
        x, W = quadrature.rule_for(wl)
        model = oracle.OracleModel(wl, x, W)
        n = wl.n
        w = np.random.default_rng(0).uniform(0, 0.05, n)
        for k in [0, 7, wl.steps - 1]:
            b = oracle.drift(model, k, n, w)
            assert abs(b + analytic.kappa_quad(wl.lam[k, n - 1], x, W)[0]) < 1e-16


def test_brownian_drift_is_lognormal_libor_drift():
    wl = workloads.tiny(N=6, driver="brownian")
    model = oracle.OracleModel(wl)
    n = wl.n
    w = np.random.default_rng(1).uniform(0, 0.1, n)
    k = 4
    lam = wl.lam[k]
    for i in range(1, n + 1):
        want = -0.5 * lam[i - 1] ** 2 - lam[i - 1] * sum(w[l - 1] * lam[l - 1] for l in range(i + 1, n + 1))
        assert abs(oracle.drift(model, k, i, w) - want) < 1e-16


def _order_slope(err_fn):
    eps = np.array([0.04, 0.02, 0.01])
    e = np.array([abs(err_fn(t)) for t in eps])
    return np.polyfit(np.log(eps), np.log(e), 1)[0]


def test_drift_expansion_error_orders():
    wl, x, W, model = _tiny(N=7, Q=24)
    n = wl.n
    lam = wl.lam[0]
    kap = lambda u: float(analytic.kappa_quad(u, x, W)[0])
    base = np.random.default_rng(3).uniform(0.5, 1.0, n)
    i = 1

    def A(t):
        return analytic.drift_jump_exact(i, t * base, lam, kap)

    s1 = _order_slope(lambda t: A(t) - analytic.drift_jump_first_order(i, t * base, lam, kap))
    s2 = _order_slope(lambda t: A(t) - analytic.drift_jump_second_order(i, t * base, lam, kap))
    s2p = _order_slope(lambda t: A(t) - analytic.drift_jump_second_order(
        i, t * base, lam, kap, printed_signs=True))
    assert abs(s1 - 2) < 0.1
    assert abs(s2 - 3) < 0.1
    # the signs as printed leave an O(|L|) error: that reading cannot be Eq. (drifta2)
    assert abs(s2p - 1) < 0.1


def test_frozen_drift_table():
    wl, x, W, model = _tiny(N=6, Q=16)
    n, S, h = wl.n, wl.steps, wl.h
    b0, D0 = oracle.frozen_drift(model)
    w0 = wl.delta * wl.L0[1:] / (1 + wl.delta * wl.L0[1:])
    for k in [0, 5, S - 1]:
        for l in range(1, n + 1):
            assert b0[k, l - 1] == oracle.drift(model, k, l, w0)
    assert np.allclose(D0[1:], np.cumsum(b0 * h, axis=0), rtol=1e-14, atol=1e-18)
    assert np.all(D0[0] == 0)
