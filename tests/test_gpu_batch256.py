"""The batched configuration at its own size: 256 independent term structures
(N from 8 to 80, uneven strike grids and path budgets, 2^24 paths in total)
in one persistent launch per scheme, replayed from a CUDA graph as the
benchmark runs it.

Instance q draws from Philox counter word 1 = q, so each instance is
checked against the FP64 oracle run with instance q:
  * prices of every instance with the smallest path budget (3957 paths, the
    2^12 budgets after the recipe's rescaling to 2^24 in total): all 35 under
    the Picard scheme (the configuration's scheme), and those with N <= 40
    under the full scheme, within 1e-7;
  * four paths sampled across every instance's budget (so they fall in
    different tiles and work items of the schedule), and 32 of the
    N = 80 instance, within 1e-5 relative on every recorded rate;
  * both under the library's default launch shape and under the one the
    bench's tuner picks for this batch (two paths per thread).
"""
import numpy as np
import pytest

from oracle import oracle as ora
from oracle import quadrature
from paper_1006_3340_gb300 import workloads

pytestmark = pytest.mark.gpu
CODES = {"picard": ora.PICARD, "full": ora.FULL}
SHAPES = (None, (128, 0, 16, 2))


@pytest.fixture(scope="module")
def lll():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1006_3340_gb300 import lll as mod

    mod.load()
    return mod


@pytest.fixture(scope="module")
def batch256(lll):
    wls = workloads.batched_instances()
    assert len(wls) == 256 and sum(wl.paths for wl in wls) == 1 << 24
    inst = [(wl,) + tuple(quadrature.rule_for(wl)) for wl in wls]
    q_long = int(np.argmax([wl.N for wl in wls]))
    counts = [32 if q == q_long else 4 for q in range(len(wls))]
    strides = [wl.paths // c for wl, c in zip(wls, counts)]
    b, keep = lll.lll_batch_init(inst)
    out = {}
    try:
        for q in range(len(wls)):
            lll.lll_batch_set_snapshots(b, q, counts[q], strides[q])
        lll.lll_batch_use_graph(b, True)
        # the library's default shape, then the one the bench's tuner picks on
        # this batch (128 threads, 16-row chunks, two paths per thread)
        for shape in SHAPES:
            if shape is not None:
                lll.lll_batch_set_launch(b, *shape)
            for scheme in ("picard", "full"):
                lll.lll_batch_simulate(b, lll.SCHEMES[scheme], 42)
                prices = [lll.lll_batch_prices(b, q, wl.n, wl.strikes.shape[1])[0] for q, wl in enumerate(wls)]
                snaps = [lll.lll_batch_get_paths(b, q, wl.n, 0, counts[q]) for q, wl in enumerate(wls)]
                out[scheme, shape] = (prices, snaps)
    finally:
        lll.lll_batch_destroy(b)
    return inst, counts, strides, q_long, out


@pytest.mark.parametrize("scheme", ["picard", "full"])
def test_smallest_budget_instances_match_oracle_prices(batch256, scheme):
    inst, _, _, _, out = batch256
    smallest = min(wl.paths for wl, _, _ in inst)
    checked = 0
    for q, (wl, x, W) in enumerate(inst):
        if wl.paths != smallest or (scheme == "full" and wl.N > 40):
            continue
        ref = ora.simulate(ora.OracleModel(wl, x, W), CODES[scheme], npaths=wl.paths, seed=42, inst=q)
        for shape in SHAPES:
            prices, _ = out[scheme, shape]
            assert np.abs(prices[q] - ref["price"]).max() <= 1e-7, (q, wl.N, shape)
        checked += 1
    assert checked == (35 if scheme == "picard" else 17)


@pytest.mark.parametrize("scheme", ["picard", "full"])
def test_sampled_paths_of_every_instance_match_oracle(batch256, scheme):
    inst, counts, strides, q_long, out = batch256
    worst = 0.0
    for q, (wl, x, W) in enumerate(inst):
        idx = np.arange(counts[q], dtype=np.uint64) * np.uint64(strides[q])
        ref = ora.simulate_paths(ora.OracleModel(wl, x, W), CODES[scheme], idx, seed=42, inst=q)
        mask = ~np.isnan(ref["snap"])
        for shape in SHAPES:
            _, snaps = out[scheme, shape]
            got = snaps[q].astype(np.float64)
            assert np.array_equal(mask, ~np.isnan(got)), (q, shape)
            rel = np.abs(np.expm1(got[mask] - ref["snap"][mask])).max()
            assert rel <= 1e-5, (q, wl.N, rel, shape)
            worst = max(worst, rel)
    assert inst[q_long][0].N == 80 and counts[q_long] == 32
