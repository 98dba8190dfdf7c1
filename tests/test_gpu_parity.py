"""GPU (liblll.so, through the C ABI) against the FP64 oracle on the same
seeded inputs and the same Philox streams.

Bar (from the arithmetic): FP32 path state over <= 476 Euler steps keeps
log-rates within ~1e-6 of FP64, so every recorded rate L_l(T_m) must agree to
1e-5 relative; caplet prices (notional 1) to 1e-7 absolute.  The IG
acceptance decision is taken in FP64 on both sides near its threshold, so no
path is excluded; the oracle's smallest margin is reported.
"""
import numpy as np
import pytest

from oracle import oracle as ora
from oracle import quadrature
from paper_1006_3340_gb300 import workloads

pytestmark = pytest.mark.gpu

REL_RATE = 1e-5
ABS_PRICE = 1e-7
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


def _compare(lll, wl, scheme, npaths, launch=None, x=None, W=None, tenor=0):
    if x is None:
        x, W = quadrature.rule_for(wl)
    sim = lll.LevyLibor(wl, x, W)
    try:
        if launch:
            sim.set_launch(*launch)
        if tenor:
            sim.set_mapping("tenor", tenor)
        sim.simulate(scheme, paths=npaths, snapshots=npaths)
        zg = sim.paths(0, npaths).astype(np.float64)
        pg, seg = sim.prices()
    finally:
        sim.close()
    ref = ora.simulate(ora.OracleModel(wl, x, W), SCHEMES[scheme], npaths=npaths, want_snap=True)
    mask = ~np.isnan(ref["snap"])
    assert np.array_equal(mask, ~np.isnan(zg))
    rel = np.abs(np.expm1(zg[mask] - ref["snap"][mask]))
    assert rel.max() <= REL_RATE, (scheme, rel.max())
    dp = np.abs(pg - ref["price"])
    assert dp.max() <= ABS_PRICE, (scheme, dp.max())
    assert np.allclose(seg, ref["se"], rtol=1e-3, atol=1e-9)
    return rel.max(), dp.max(), ref["min_margin"].min()


@pytest.mark.parametrize("scheme", ["full", "picard", "frozen"])
def test_small_plain(lll, scheme):
    wl = workloads.small_plain(paths=4000)  # 31.25 blocks of 128: ragged last tile
    _compare(lll, wl, scheme, 4000)


@pytest.mark.parametrize("scheme", ["full", "picard"])
def test_small_plain_brownian(lll, scheme):
    wl = workloads.small_plain(paths=3000, driver="brownian")
    _compare(lll, wl, scheme, 3000)


@pytest.mark.parametrize("scheme", ["full", "picard", "frozen"])
def test_large_single_subset(lll, scheme):
    wl = workloads.large_single()
    _compare(lll, wl, scheme, 2048 + 37)


@pytest.mark.parametrize("scheme", ["full", "picard"])
def test_long_dated_subset(lll, scheme):
    wl = workloads.long_dated()
    _compare(lll, wl, scheme, 200)


@pytest.mark.parametrize("N,s,Q,paths", [(2, 1, 8, 1), (3, 2, 8, 33), (5, 3, 20, 200), (7, 4, 40, 129)])
@pytest.mark.parametrize("scheme", ["full", "picard", "frozen"])
@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_tiny_edge_shapes(lll, N, s, Q, paths, scheme, lanes):
    wl = workloads.tiny(N=N, s=s, Q=Q, paths=paths)
    _compare(lll, wl, scheme, paths, launch=(0, 0, 0, 0, lanes if scheme != "frozen" else 1))


@pytest.mark.parametrize("launch", [(32, 0, 1, 1, 1), (64, 1, 2, 2, 1), (256, 0, 3, 1, 1), (96, 2, 0, 2, 1),
                                    (128, 0, 0, 1, 1), (256, 0, 0, 2, 1), (32, 0, 1, 0, 4), (64, 1, 2, 0, 4),
                                    (256, 0, 3, 0, 4), (96, 2, 0, 0, 4), (128, 0, 0, 0, 4), (64, 0, 3, 0, 2),
                                    (128, 0, 0, 0, 2)])
def test_launch_shapes_agree(lll, launch):
    wl = workloads.large_single()
    _compare(lll, wl, "picard", 300, launch=launch)


# Tenor-parallel mapping (lll_set_mapping): G lanes per path, each owning a
# block of rates; shapes where the last lanes own fewer rates or none (n=39,
# G=16 gives r=3 and 13 busy lanes; n=9, G=32), ragged path tiles, one path.
@pytest.mark.parametrize("lanes", [4, 8, 16, 32])
@pytest.mark.parametrize("scheme", ["full", "picard"])
def test_tenor_mapping_large_single(lll, scheme, lanes):
    wl = workloads.large_single()
    _compare(lll, wl, scheme, 1000 + 37, tenor=lanes)


@pytest.mark.parametrize("lanes", [4, 32])
@pytest.mark.parametrize("scheme", ["full", "picard"])
def test_tenor_mapping_small_plain(lll, scheme, lanes):
    wl = workloads.small_plain(paths=3001)
    _compare(lll, wl, scheme, 3001, tenor=lanes)


@pytest.mark.parametrize("N,s,Q,paths", [(2, 1, 8, 1), (3, 2, 8, 33), (7, 4, 40, 129)])
@pytest.mark.parametrize("lanes", [4, 8])
def test_tenor_mapping_tiny_edge_shapes(lll, N, s, Q, paths, lanes):
    wl = workloads.tiny(N=N, s=s, Q=Q, paths=paths)
    for scheme in ("full", "picard"):
        _compare(lll, wl, scheme, paths, tenor=lanes)


@pytest.mark.parametrize("scheme", ["full", "picard"])
def test_tenor_mapping_long_dated(lll, scheme):
    wl = workloads.long_dated()
    _compare(lll, wl, scheme, 100, tenor=8)


def test_tenor_mapping_refuses_swaptions_and_keeps_other_schemes(lll):
    wl = workloads.small_plain(paths=500)
    x, W = quadrature.rule_for(wl)
    sim = lll.LevyLibor(wl, x, W)
    try:
        sim.set_mapping("tenor", 8)
        sim.simulate("frozen")  # frozen drift keeps the path kernel
        sim.set_product("swaption")
        with pytest.raises(lll.LLLError) as e:
            sim.simulate("picard")
        assert e.value.code == lll.LLL_EUNSUPPORTED
        sim.set_mapping("path")
        sim.simulate("picard")
    finally:
        sim.close()


# Step-parallel mapping of the Picard scheme (lll_set_mapping("step")): the
# Euler steps of a path evaluated in parallel from prefix sums of lambda dH.
@pytest.mark.parametrize("maker,paths", [(workloads.small_plain, 3001), (workloads.large_single, 1037),
                                         (workloads.long_dated, 100)])
def test_step_mapping_picard_matches_oracle(lll, maker, paths):
    wl = maker(paths=paths) if maker is not workloads.large_single else maker()
    x, W = quadrature.rule_for(wl)
    sim = lll.LevyLibor(wl, x, W)
    try:
        sim.set_mapping("step")
        sim.simulate("picard", paths=paths, snapshots=paths)
        zg = sim.paths(0, paths).astype(np.float64)
        pg, _ = sim.prices()
    finally:
        sim.close()
    ref = ora.simulate(ora.OracleModel(wl, x, W), ora.PICARD, npaths=paths, want_snap=True)
    mask = ~np.isnan(ref["snap"])
    assert np.array_equal(mask, ~np.isnan(zg))
    assert np.abs(np.expm1(zg[mask] - ref["snap"][mask])).max() <= REL_RATE
    assert np.abs(pg - ref["price"]).max() <= ABS_PRICE


@pytest.mark.parametrize("N,s,Q,paths", [(2, 1, 8, 1), (3, 2, 8, 33), (7, 4, 40, 129)])
def test_step_mapping_tiny_edge_shapes(lll, N, s, Q, paths):
    wl = workloads.tiny(N=N, s=s, Q=Q, paths=paths)
    x, W = quadrature.rule_for(wl)
    sim = lll.LevyLibor(wl, x, W)
    try:
        sim.set_mapping("step")
        sim.simulate("picard", paths=paths, snapshots=paths)
        zg = sim.paths(0, paths).astype(np.float64)
        pg, _ = sim.prices()
    finally:
        sim.close()
    ref = ora.simulate(ora.OracleModel(wl, x, W), ora.PICARD, npaths=paths, want_snap=True)
    mask = ~np.isnan(ref["snap"])
    assert np.abs(np.expm1(zg[mask] - ref["snap"][mask])).max() <= REL_RATE
    assert np.abs(pg - ref["price"]).max() <= ABS_PRICE


def test_step_mapping_equals_path_mapping_across_chunks(lll):
    """50,001 paths of the N=40 workload take three chunks of the step-parallel
    pipeline (20,480 paths each).  Each unit does the path kernel's arithmetic
    in the same order, so every recorded log-rate is bit-equal to the path
    mapping's and the prices differ only by the payoff reduction order."""
    wl = workloads.large_single(paths=50001)
    x, W = quadrature.rule_for(wl)
    sim = lll.LevyLibor(wl, x, W)
    try:
        sim.set_launch(128, 0, 0, 1, 1)
        sim.simulate("picard", snapshots=200, snapshot_stride=250)
        z_path = sim.paths(0, 200)
        p_path, _ = sim.prices()
        sim.set_mapping("step")
        sim.simulate("picard", snapshots=200, snapshot_stride=250)
        z_step = sim.paths(0, 200)
        p_step, _ = sim.prices()
        with pytest.raises(lll.LLLError) as e:
            sim.simulate("full")
        assert e.value.code == lll.LLL_EUNSUPPORTED
    finally:
        sim.close()
    mask = ~np.isnan(z_path)
    assert np.array_equal(z_path[mask], z_step[mask])
    assert np.allclose(p_step, p_path, rtol=1e-12, atol=1e-18)
