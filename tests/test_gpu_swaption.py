"""Co-terminal payer swaptions (lll_set_product(LLL_PRODUCT_SWAPTION)) on the
same simulated paths as the caplets.

* Against the FP64 oracle: the oracle's swaption prices (oracle.swaption_prices,
  bond prices at each expiry from its own log-rates of the same Philox paths)
  must equal the GPU's within 1e-7 for the quadrature schemes.
* At the last expiry the swap has one period, so the swaption is the last
  caplet: equal prices on the same paths (to the FP32 rounding of the caplet
  payoff).
* With strike 0 the payoff is 1 / B(T_m, T_N) - 1, whose expectation under the
  terminal measure is B(0,T_m) / B(0,T_N) - 1: the price must equal
  B(0,T_m) - B(0,T_N) within three standard errors (a property of the model,
  independent of the payoff code).
"""
import numpy as np
import pytest

from oracle import oracle as ora
from oracle import quadrature
from paper_1006_3340_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lll():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1006_3340_gb300 import lll as mod

    mod.load()
    return mod


@pytest.mark.parametrize("scheme,code", [("full", ora.FULL), ("picard", ora.PICARD)])
def test_swaptions_match_oracle_paths(lll, scheme, code):
    wl = workloads.large_single(paths=2048)
    x, W = quadrature.rule_for(wl)
    sim = lll.LevyLibor(wl, x, W)
    try:
        sim.set_product("swaption")
        sim.simulate(scheme)
        p, _ = sim.prices()
    finally:
        sim.close()
    ref = ora.simulate(ora.OracleModel(wl, x, W), code, want_snap=True)
    want = ora.swaption_prices(wl, ref["snap"], wl.strikes)
    assert np.abs(p - want).max() <= 1e-7


def test_last_expiry_swaption_is_last_caplet(lll):
    wl = workloads.small_plain(paths=20000)
    sim = lll.LevyLibor(wl)
    try:
        sim.simulate("full")
        cap, _ = sim.prices()
        sim.set_product("swaption")
        sim.simulate("full")
        swp, _ = sim.prices()
    finally:
        sim.close()
    # the caplet payoff is formed in FP32, the swaption's in FP64: equal to FP32 rounding
    assert np.allclose(swp[-1], cap[-1], rtol=1e-6, atol=1e-14)
    assert np.all(swp[:-1] > cap[:-1])  # a co-terminal swaption with a longer swap is worth more


@pytest.mark.parametrize("scheme", ["full", "picard", "mlp"])
def test_zero_strike_swaption_is_forward_bond_value(lll, scheme):
    wl = workloads.large_single(paths=1 << 16)
    wl = wl.with_paths(1 << 16)
    x, W = quadrature.rule_for(wl)
    sim = lll.LevyLibor(wl, x, W)
    try:
        if scheme == "mlp":
            lll.lll_mlp_train(sim.ctx, hidden=128, layers=3, train_paths=1 << 14, records_per_path=4,
                              epochs=2, batch=4096, lr=2e-3, lr_final=2e-4, seed=3)
        sim.set_strikes(np.zeros((wl.n, 1)))
        sim.set_product("swaption")
        sim.simulate(scheme)
        p, se = sim.prices()
    finally:
        sim.close()
    want = np.array([ora.discount(wl, m) - ora.discount_terminal(wl) for m in range(1, wl.n + 1)])
    assert np.all(np.abs(p[:, 0] - want) <= 3 * se[:, 0] + 1e-12), np.max(np.abs(p[:, 0] - want) / se[:, 0])
