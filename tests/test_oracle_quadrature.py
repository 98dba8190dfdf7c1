"""Pins of the oracle's Gauss rule for x^2 nu(x) dx on [-a, a].

  * Gauss exactness: for every polynomial p of degree <= 2Q-1 the rule
    reproduces int p m dx, with the integral taken by scipy's adaptive
    quadrature of the closed-form weight (Legendre basis in x/a keeps the
    comparison well-conditioned).
  * The rule's jump cumulant plus the tail integral beyond a equals the
    closed-form NIG cumulant kappa(u) (Section 4), which ties the Levy density
    used to build the rule to the paper's kappa.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special

from oracle import analytic, quadrature
from paper_1006_3340_gb300 import workloads

CASES = [(18.0, -4.0, 1.0, 1.5), (12.0, -3.0, 0.8, 1.5), (10.0, -2.5, 1.2, 1.5),
         (9.0, -2.0, 1.0, 1.5)]


@pytest.mark.parametrize("alpha,beta,dbar,a", CASES)
@pytest.mark.parametrize("Q", [8, 32])
def test_gauss_exactness(alpha, beta, dbar, a, Q):
    x, W = quadrature.gauss_rule(alpha, beta, dbar, a, Q)
    assert np.all(W > 0) and np.all(np.abs(x) < a) and np.all(np.diff(x) > 0)
    m = lambda t: float(quadrature.x2nu(t, alpha, beta, dbar))
    for r in range(0, 2 * Q):
        Pr = scipy.special.legendre(r)
        exact = scipy.integrate.quad(lambda t: Pr(t / a) * m(t), -a, a, points=[0.0],
                                     epsabs=1e-15, epsrel=1e-13, limit=500)[0]
        got = float(np.sum(W * Pr(x / a)))
        scale = scipy.integrate.quad(lambda t: abs(Pr(t / a)) * m(t), -a, a, points=[0.0],
                                     limit=500)[0]
        assert abs(got - exact) < 1e-11 * scale, (r, got, exact)


@pytest.mark.parametrize("alpha,beta,dbar,a", CASES)
def test_rule_reproduces_nig_cumulant(alpha, beta, dbar, a):
    Q = 32
    x, W = quadrature.gauss_rule(alpha, beta, dbar, a, Q)
    g = math.sqrt(alpha ** 2 - beta ** 2)
    mu = -dbar * beta / g  # martingale drift: kappa(u) = int (e^{ux}-1-ux) nu(dx)
    for u in [-0.3, -0.15, 0.05, 0.12, 0.25, 0.4]:
        kq = float(analytic.kappa_quad(u, x, W)[0])
        tail = analytic.kappa_tail(u, alpha, beta, dbar, a)
        ex = float(analytic.kappa(u, alpha, beta, dbar, mu))
        assert abs(kq + tail - ex) < 1e-10 * abs(ex), (u, kq, tail, ex)


def test_total_mass_is_truncated_variance():
    # sum W = int_{|x|<=a} x^2 nu = kappa''(0) minus the tail's second moment
    alpha, beta, dbar, a = 12.0, -3.0, 0.8, 1.5
    x, W = quadrature.gauss_rule(alpha, beta, dbar, a, 64)
    g = math.sqrt(alpha ** 2 - beta ** 2)
    var = dbar * alpha ** 2 / g ** 3
    f = lambda t: t * t * float(quadrature.levy_density(t, alpha, beta, dbar))
    tail = scipy.integrate.quad(f, a, np.inf)[0] + scipy.integrate.quad(f, -np.inf, -a)[0]
    assert abs(W.sum() + tail - var) < 1e-10 * var


def test_symmetric_measure_gives_symmetric_rule():
    x, W = quadrature.gauss_rule(1.5, 0.0, 1.5, 30.0, 24)
    assert np.allclose(x, -x[::-1], atol=1e-12 * 30)
    assert np.allclose(W, W[::-1], rtol=1e-10)


def test_workload_rules_are_well_formed():
    for wl in [workloads.small_plain(), workloads.large_single(), workloads.long_dated()]:
        x, W = quadrature.rule_for(wl)
        assert len(x) == wl.Q and np.all(x != 0) and np.all(W > 0)
