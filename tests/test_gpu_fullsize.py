"""Full-size runs (the launch shapes the benchmark times) checked on sampled
outputs and on properties that hold at any size.

  * Paths sampled across the whole 2^20-path range of the N=40 workload (and
    the 2^22-path N=120 workload) agree with the oracle computed path by path.
  * A zero-strike caplet pays delta L_m(T_m) prod_{l>m}(1 + delta L_l(T_m)) =
    prod_{l>=m}(...) - prod_{l>m}(...); both products are deflated bond
    prices (martingales under the terminal measure), so its price is the FRA
    value B(0,T_m) - B(0,T_{m+1}) (Eq. (caplet) with K = 0).
  * Results are run-to-run deterministic, and path shards merge to the
    unsharded sums (Philox counters are keyed by the global path index).
"""
import numpy as np
import pytest

from oracle import oracle as ora
from oracle import quadrature
from paper_1006_3340_gb300 import workloads

pytestmark = pytest.mark.gpu
SCHEMES = {"full": ora.FULL, "picard": ora.PICARD, "frozen": ora.FROZEN}


@pytest.fixture(scope="module")
def lll():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1006_3340_gb300 import lll as mod

    mod.load()
    return mod


@pytest.mark.parametrize("maker,scheme,stride", [
    (workloads.large_single, "picard", 4096),
    (workloads.large_single, "full", 4096),
    (workloads.long_dated, "picard", 1 << 16),
])
def test_sampled_paths_at_full_size(lll, maker, scheme, stride):
    wl = maker()
    x, W = quadrature.rule_for(wl)
    count = wl.paths // stride
    sim = lll.LevyLibor(wl, x, W)
    try:
        sim.simulate(scheme, snapshots=count, snapshot_stride=stride)
        zg = sim.paths(0, count).astype(np.float64)
    finally:
        sim.close()
    idx = np.arange(count, dtype=np.uint64) * stride
    ref = ora.simulate_paths(ora.OracleModel(wl, x, W), SCHEMES[scheme], idx)
    mask = ~np.isnan(ref["snap"])
    rel = np.abs(np.expm1(zg[mask] - ref["snap"][mask]))
    assert rel.max() <= 1e-5, rel.max()


@pytest.mark.parametrize("scheme", ["full", "picard"])
def test_zero_strike_caplets_are_fra_values(lll, scheme):
    wl = workloads.large_single()
    n = wl.n
    strikes = np.zeros((n, 1))
    sim = lll.LevyLibor(wl)
    try:
        sim.set_strikes(strikes)
        sim.simulate(scheme)
        p, se = sim.prices()
    finally:
        sim.close()
    for m in range(1, n + 1):
        fra = ora.discount(wl, m) - ora.discount(wl, m + 1)
        assert abs(p[m - 1, 0] - fra) < 4 * se[m - 1, 0] + 2e-6 * fra, (m, p[m - 1, 0], fra, se[m - 1, 0])


def test_deterministic_and_shards_merge(lll):
    wl = workloads.large_single(paths=1 << 18)
    sim = lll.LevyLibor(wl)
    try:
        sim.simulate("picard")
        a1, a2, na = sim.sums()
        sim.simulate("picard")
        b1, b2, _ = sim.sums()
        assert np.array_equal(a1, b1) and np.array_equal(a2, b2)
        half = wl.paths // 2 + 77
        sim.simulate("picard", paths=half, first_path=0)
        c1, c2, nc = sim.sums()
        sim.simulate("picard", paths=wl.paths - half, first_path=half)
        d1, d2, nd = sim.sums()
        assert nc + nd == na
        assert np.allclose(c1 + d1, a1, rtol=1e-12, atol=0)
        assert np.allclose(c2 + d2, a2, rtol=1e-12, atol=0)
    finally:
        sim.close()
