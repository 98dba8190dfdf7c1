"""Pins of the oracle's schemes and caplet prices (Eq. (caplet)).

  * Brownian driver: the log-normal LIBOR model prices caplets by Black's
    formula (Section 1); full and Picard Monte Carlo within 3 standard errors.
  * Last rate: driftless under the terminal measure, so its caplet is an
    exponential-NIG option; Fourier inversion and direct density integration
    agree to 1e-8, and the Monte Carlo matches within 3 standard errors.
  * Deflated bonds: E[prod_{l>=i}(1 + delta L_l(T_i))] = B(0,T_i)/B(0,T_N)
    (B(t,T_i)/B(t,T_N) is a martingale under the terminal measure).
  * Picard structure (Eq. (Picard-2), (bdrift)): the last rate has a
    deterministic drift, so Z^(1) of the last rate is exact; hence the Picard
    scheme reproduces the full scheme exactly on the last two rates and
    differs from the third-last on.  The frozen drift reproduces only the
    last rate.
  * Approximation orders: under L(0) -> eps L(0) the pathwise Picard error
    shrinks like eps^2 and the frozen-drift error like eps.
"""
import math

import numpy as np
import pytest

from oracle import analytic, oracle, quadrature
from paper_1006_3340_gb300 import workloads


def _run(wl, scheme, **kw):
    x, W = quadrature.rule_for(wl)
    return oracle.simulate(oracle.OracleModel(wl, x, W), scheme, **kw)


@pytest.mark.parametrize("scheme", [oracle.FULL, oracle.PICARD])
def test_brownian_caplets_match_black(scheme):
    wl = workloads.small_plain(paths=20000, driver="brownian")
    r = _run(wl, scheme)
    n = wl.n
    for m in range(1, n + 1):
        T = m * wl.delta
        sigma = math.sqrt(np.mean(wl.lam[: m * wl.s, m - 1] ** 2))
        K = wl.strikes[m - 1, 0]
        B_pay = oracle.discount(wl, m + 1)
        bl = analytic.black_caplet(wl.L0[m], K, sigma, T, wl.delta, B_pay)
        assert abs(r["price"][m - 1, 0] - bl) < 3 * r["se"][m - 1, 0], (m, r["price"][m - 1, 0], bl)


def test_last_caplet_fourier_equals_density():
    wl = workloads.small_plain()
    x, W = quadrature.rule_for(wl)
    for K in [0.03, 0.04, 0.05]:
        f = analytic.last_caplet_fourier(wl, x, W, K)
        d = analytic.last_caplet_density(wl, x, W, K)
        assert abs(f - d) < 1e-8, (K, f, d)


@pytest.mark.parametrize("maker,scheme", [(workloads.small_plain, oracle.FULL),
                                          (workloads.small_plain, oracle.PICARD),
                                          (workloads.large_single, oracle.FULL)])
def test_last_caplet_monte_carlo_matches_fourier(maker, scheme):
    wl = maker(paths=20000 if maker is workloads.small_plain else 4096)
    x, W = quadrature.rule_for(wl)
    r = oracle.simulate(oracle.OracleModel(wl, x, W), scheme)
    n = wl.n
    atm = analytic.last_caplet_fourier(wl, x, W, wl.L0[n])
    checked = 0
    for q in range(wl.strikes.shape[1]):
        K = wl.strikes[n - 1, q]
        f = analytic.last_caplet_fourier(wl, x, W, K)
        if f < 0.05 * atm:  # too few in-the-money paths for a standard error
            continue
        checked += 1
        assert abs(r["price"][n - 1, q] - f) < 3 * r["se"][n - 1, q], (q, r["price"][n - 1, q], f)
    assert checked >= 1


@pytest.mark.parametrize("scheme", [oracle.FULL, oracle.PICARD])
def test_deflated_bonds(scheme):
    wl = workloads.small_plain(paths=20000)
    r = _run(wl, scheme, want_snap=True)
    snap = r["snap"]
    n = wl.n
    BN = oracle.discount_terminal(wl)
    for m in range(1, n + 1):
        L = np.exp(snap[:, m - 1, m - 1:])
        prod = np.prod(1 + wl.delta * L, axis=1)
        want = oracle.discount(wl, m) / BN
        se = prod.std(ddof=1) / math.sqrt(len(prod))
        assert abs(prod.mean() - want) < 3 * se + 2e-6 * want, (m, prod.mean(), want, se)


def test_picard_exact_on_last_two_rates():
    wl = workloads.large_single(paths=64)
    x, W = quadrature.rule_for(wl)
    model = oracle.OracleModel(wl, x, W)
    full = oracle.simulate(model, oracle.FULL, want_snap=True)["snap"]
    pic = oracle.simulate(model, oracle.PICARD, want_snap=True)["snap"]
    frz = oracle.simulate(model, oracle.FROZEN, want_snap=True)["snap"]
    n = wl.n
    for m in range(1, n + 1):
        d_pic = np.abs(pic[:, m - 1, m - 1:] - full[:, m - 1, m - 1:])
        d_frz = np.abs(frz[:, m - 1, m - 1:] - full[:, m - 1, m - 1:])
        assert np.all(d_pic[:, -2:] < 1e-12)          # rates n-1, n
        assert np.all(d_frz[:, -1] < 1e-12)           # rate n
        if m <= n - 2:
            assert np.max(d_pic[:, :-2]) > 1e-12     # rates m..n-2 differ
        if m <= n - 1:
            assert np.max(d_frz[:, :-1]) > 1e-12


def test_picard_and_frozen_error_orders():
    base = workloads.large_single(paths=32)
    x, W = quadrature.rule_for(base)
    errs = {oracle.PICARD: [], oracle.FROZEN: []}
    eps = [1.0, 0.5, 0.25]
    for e in eps:
        wl = workloads.large_single(paths=32)
        wl.L0 = base.L0 * e
        wl.strikes = base.strikes * e
        model = oracle.OracleModel(wl, x, W)
        full = oracle.simulate(model, oracle.FULL, want_snap=True)["snap"]
        for sch in errs:
            snap = oracle.simulate(model, sch, want_snap=True)["snap"]
            errs[sch].append(np.nanmax(np.abs(snap - full)))
    sp = np.polyfit(np.log(eps), np.log(errs[oracle.PICARD]), 1)[0]
    sf = np.polyfit(np.log(eps), np.log(errs[oracle.FROZEN]), 1)[0]
    assert abs(sp - 2) < 0.25, errs
    assert abs(sf - 1) < 0.25, errs
    assert errs[oracle.PICARD][0] < 0.1 * errs[oracle.FROZEN][0]


def test_schemes_share_random_numbers_and_are_deterministic():
    wl = workloads.small_plain(paths=500)
    a = _run(wl, oracle.PICARD, threads=1)
    b = _run(wl, oracle.PICARD, threads=7)
    assert np.allclose(a["sum"], b["sum"], rtol=1e-13, atol=0)
    c = _run(wl, oracle.PICARD, threads=7)
    assert np.array_equal(b["sum"], c["sum"])


def test_swaption_oracle_last_expiry_is_last_caplet_and_zero_strike_is_forward_bond():
    """A co-terminal swaption with one period left is the last caplet on the
    same paths; with strike 0 its deflated payoff is 1 / B(T_m, T_N) - 1,
    whose terminal-measure mean is B(0, T_m) / B(0, T_N) - 1 (deflated bond
    prices are martingales), so the price is B(0, T_m) - B(0, T_N)."""
    wl = workloads.small_plain(paths=20000)
    x, W = quadrature.rule_for(wl)
    r = oracle.simulate(oracle.OracleModel(wl, x, W), oracle.FULL, want_snap=True)
    swp = oracle.swaption_prices(wl, r["snap"], wl.strikes)
    assert abs(swp[-1, 0] - r["price"][-1, 0]) <= 1e-15
    assert np.all(swp[:-1, 0] > r["price"][:-1, 0])
    zero = oracle.swaption_prices(wl, r["snap"], np.zeros((wl.n, 1)))[:, 0]
    want = np.array([oracle.discount(wl, m) - oracle.discount_terminal(wl) for m in range(1, wl.n + 1)])
    # the same path average of B(0,T_N) (prod_{l>=m}(1 + delta L_l) - 1): compare
    # against its standard error
    BN = oracle.discount_terminal(wl)
    for m in range(1, wl.n + 1):
        L = np.exp(r["snap"][:, m - 1, m - 1:])
        v = BN * (np.prod(1.0 + wl.delta * L, axis=1) - 1.0)
        assert abs(zero[m - 1] - v.mean()) <= 1e-14
        assert abs(zero[m - 1] - want[m - 1]) <= 3 * v.std() / np.sqrt(len(v)), m
