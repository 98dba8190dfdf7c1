"""Pins of the drift-expansion schemes (oracle/expansion.py, Eq. (drifta) and
Eq. (drifta2)).

* The vectorised A' and A'' equal the per-rate formulas of oracle/analytic.py,
  which the error-order test of test_oracle_drift.py pins to the exact
  inclusion-exclusion drift (errors O(|L|^2) and O(|L|^3)).
* With the quadrature rule's own cumulant the expansions are truncations of
  the oracle's full-scheme compensator: the first order is exact when each
  rate has at most one later rate (N = 3), the second order when it has at
  most two (N = 4).  The schemes must then reproduce the C oracle's full
  scheme path by path.
* The paper's numerical example (Section 4): with the NIG cumulant the
  implied-volatility errors of the two expansions against the full SDE are
  printed as average 0.41 bp / max 9.5 bp (first order) and 0.013 / 0.38 bp
  (second order) (tests/golden/paper_section4_example.txt).  The strike grid
  is not printed; on ATM +- 150 bp the reproduction must land within a factor
  of three of each, with the second order far below the first.
"""
import os

import numpy as np

from oracle import analytic, expansion, oracle, quadrature
from paper_1006_3340_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_section4_example.txt")


def test_vectorised_expansions_equal_per_rate_formulas():
    wl = workloads.tiny(N=7, Q=24)
    x, W = quadrature.rule_for(wl)
    kap = lambda u: analytic.kappa_quad(u, x, W)
    lam = np.asarray(wl.lam)[2]
    n = len(lam)
    rng = np.random.default_rng(4)
    w = rng.uniform(0.0, 0.05, size=(5, n))
    for order in (1, 2):
        A = expansion.drift(w, *expansion.drift_terms(lam, kap, order))
        for p in range(5):
            for i in range(1, n + 1):
                f = analytic.drift_jump_first_order if order == 1 else analytic.drift_jump_second_order
                ref = f(i, w[p], lam, lambda u: float(kap(u)[0]))
                assert abs(A[p, i - 1] - ref) <= 1e-15 + 1e-12 * abs(ref)


def _vs_full(N, order):
    wl = workloads.tiny(N=N, s=4, Q=16, paths=32)
    x, W = quadrature.rule_for(wl)
    model = oracle.OracleModel(wl, x, W)
    got = expansion.simulate_expansion(model, order, lambda u: analytic.kappa_quad(u, x, W))
    ref = oracle.simulate(model, oracle.FULL, want_snap=True)
    mask = ~np.isnan(ref["snap"])
    return np.abs(got["snap"][mask] - ref["snap"][mask]).max(), np.abs(got["price"] - ref["price"]).max()


def test_first_order_is_exact_with_one_later_rate():
    dz, dp = _vs_full(3, 1)
    assert dz <= 1e-12 and dp <= 1e-14


def test_second_order_is_exact_with_two_later_rates():
    dz, dp = _vs_full(4, 2)
    assert dz <= 1e-12 and dp <= 1e-14
    dz1, _ = _vs_full(4, 1)  # the first order is not
    assert dz1 > 1e-9


def test_paper_example_expansion_errors_reproduce_section_4():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    printed = {r[1]: (float(r[2]), float(r[3])) for r in rows if r[0] == "IV_BP"}
    wl = workloads.paper_example(paths=10000, offsets_bp=(-150, -100, -50, 0, 50, 100, 150))
    x, W = quadrature.rule_for(wl)
    model = oracle.OracleModel(wl, x, W)
    full = oracle.simulate(model, oracle.FULL)["price"]
    kap = lambda u: analytic.kappa_wl(u, wl)
    gaps = {}
    for order, name in ((1, "first_order"), (2, "second_order")):
        p = expansion.simulate_expansion(model, order, kap)["price"]
        g = []
        for m in range(1, wl.n + 1):
            for q in range(wl.strikes.shape[1]):
                args = (wl.L0[m], wl.strikes[m - 1, q], m * wl.delta, wl.delta, oracle.discount(wl, m + 1))
                g.append(1e4 * (analytic.black_implied_vol(p[m - 1, q], *args)
                                - analytic.black_implied_vol(full[m - 1, q], *args)))
        g = np.abs(np.array(g))
        g = g[~np.isnan(g)]
        gaps[name] = (g.mean(), g.max())
    for name, (avg, mx) in gaps.items():
        pa, pm = printed[name]
        assert pa / 3 < avg < pa * 3, (name, avg, pa)
        assert pm / 3 < mx < pm * 3, (name, mx, pm)
    assert gaps["second_order"][1] < 0.1 * gaps["first_order"][1]
