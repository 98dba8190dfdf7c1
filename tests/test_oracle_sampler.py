"""Pins of the oracle's driver increments (Section 4: NIG via inverse-Gaussian
subordination, IG by Michael-Schucany-Haas; Brownian variant).

Pins: the NIG cumulants per step (derivatives of kappa at 0, times h), a KS
test against scipy's independent NIG distribution, normality of the Brownian
increment, and the acceptance-margin statistics.
"""
import math

import numpy as np
import pytest
import scipy.stats

from oracle import oracle
from paper_1006_3340_gb300 import workloads


def _cumulants(x):
    m = x.mean()
    c = x - m
    k2 = (c ** 2).mean()
    k3 = (c ** 3).mean()
    k4 = (c ** 4).mean() - 3 * k2 ** 2
    return m, k2, k3, k4


def _nig_cumulants_per_step(wl, order=8):
    """kappa_r = r! [u^r] of h * dbar (gamma - sqrt(alpha^2 - (beta+u)^2)), r >= 2,
    from the binomial series of sqrt(A (1 + t)), t = (-2 beta u - u^2) / A."""
    from numpy.polynomial import polynomial as P
    a, b, d, h = wl.alpha, wl.beta, wl.dbar, wl.h
    A = a * a - b * b
    t = np.array([0.0, -2 * b / A, -1.0 / A])
    series = np.zeros(order + 1)
    tk = np.array([1.0])
    coef = 1.0
    for k in range(order + 1):
        if k > 0:
            coef *= (0.5 - (k - 1)) / k
            tk = P.polymul(tk, t)[: order + 1]
        series[: len(tk)] += coef * tk
    kap = -d * h * math.sqrt(A) * series
    return {r: math.factorial(r) * kap[r] for r in range(2, order + 1)}


@pytest.mark.parametrize("maker", [workloads.large_single, workloads.small_plain])
def test_nig_increment_cumulants(maker):
    wl = maker(paths=4096)
    model = oracle.OracleModel(wl, np.ones(1), np.ones(1))
    dH, _ = oracle.increments(model, 0, 2048)
    x = dH.ravel()
    N = x.size
    k = _nig_cumulants_per_step(wl)
    g = math.sqrt(wl.alpha ** 2 - wl.beta ** 2)
    # closed forms of the first three jump cumulants pin the series helper itself
    assert abs(k[2] / (wl.dbar * wl.alpha ** 2 / g ** 3 * wl.h) - 1) < 1e-12
    assert abs(k[3] / (3 * wl.dbar * wl.alpha ** 2 * wl.beta / g ** 5 * wl.h) - 1) < 1e-12
    assert abs(k[4] / (3 * wl.dbar * wl.alpha ** 2 * (wl.alpha ** 2 + 4 * wl.beta ** 2)
                       / g ** 7 * wl.h) - 1) < 1e-12
    m, s2, s3, s4 = _cumulants(x)
    # large-sample standard errors of the sample cumulants (Kendall & Stuart)
    se_m = math.sqrt(k[2] / N)
    se2 = math.sqrt((k[4] + 2 * k[2] ** 2) / N)
    se3 = math.sqrt((k[6] + 9 * k[4] * k[2] + 9 * k[3] ** 2 + 6 * k[2] ** 3) / N)
    se4 = math.sqrt((k[8] + 16 * k[6] * k[2] + 48 * k[5] * k[3] + 34 * k[4] ** 2
                     + 72 * k[4] * k[2] ** 2 + 144 * k[3] ** 2 * k[2] + 24 * k[2] ** 4) / N)
    assert abs(m) < 5 * se_m
    assert abs(s2 - k[2]) < 5 * se2
    assert abs(s3 - k[3]) < 5 * se3
    assert abs(s4 - k[4]) < 5 * se4
    # the checks must be able to see a wrong variance (e.g. dbar^2 for dbar)
    assert 5 * se2 < 0.2 * k[2]


def test_nig_increment_ks_against_scipy():
    wl = workloads.large_single(paths=4096)
    model = oracle.OracleModel(wl, np.ones(1), np.ones(1))
    dH, _ = oracle.increments(model, 100, 64)
    x = dH.ravel()[:20000]
    h = wl.h
    d = wl.dbar * h
    g = math.sqrt(wl.alpha ** 2 - wl.beta ** 2)
    mu = -wl.dbar * wl.beta / g * h
    # scipy's norminvgauss(a, b, loc, scale) is NIG(alpha=a/scale, beta=b/scale, delta=scale, mu=loc)
    dist = scipy.stats.norminvgauss(wl.alpha * d, wl.beta * d, loc=mu, scale=d)
    p = scipy.stats.kstest(x, dist.cdf).pvalue
    assert p > 1e-3


def test_brownian_increment_is_normal():
    wl = workloads.small_plain(paths=1000, driver="brownian")
    model = oracle.OracleModel(wl)
    dH, mg = oracle.increments(model, 0, 300)
    z = dH.ravel() / math.sqrt(wl.h)
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-3
    assert np.all(np.isinf(mg))


def test_acceptance_margin_density():
    # u2 is uniform and independent of the threshold, so P(|margin| < e) ~ 2e.
    wl = workloads.large_single(paths=4096)
    model = oracle.OracleModel(wl, np.ones(1), np.ones(1))
    _, mg = oracle.increments(model, 0, 256)
    frac = np.mean(np.abs(mg) < 1e-3)
    assert abs(frac - 2e-3) < 5 * math.sqrt(2e-3 / mg.size)


def test_increments_depend_only_on_counter():
    wl = workloads.large_single(paths=4096)
    model = oracle.OracleModel(wl, np.ones(1), np.ones(1))
    a, _ = oracle.increments(model, 10, 4)
    b, _ = oracle.increments(model, 12, 1)
    assert np.array_equal(a[2], b[0])
    c, _ = oracle.increments(model, 10, 4, inst=1)
    assert not np.any(a == c)
