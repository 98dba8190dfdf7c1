"""Batched uneven term structures in one persistent launch (lll_batch_*).

Each instance q draws from its own Philox stream (counter word 1 = q), so it
is checked against the FP64 oracle run with instance q: prices within 1e-7.
The CUDA-graph replay must reproduce the eager launch exactly (the blocks
claim work items from a counter, in whatever order they get to it, and the
results must not depend on it), and the schedule must give the same sums
whatever the launch shape (within FP64 rounding of the different grouping of
the partial sums).
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


def _instances(count, total_paths, seed=5):
    out = []
    for wl in workloads.batched_instances(n_inst=count, total_paths=total_paths, seed=seed):
        wl = wl.with_paths(max(wl.paths, 1))
        x, W = quadrature.rule_for(wl)
        out.append((wl, x, W))
    return out


def _prices(lll, b, inst):
    return [lll.lll_batch_prices(b, q, wl.n, wl.strikes.shape[1]) for q, (wl, _, _) in enumerate(inst)]


@pytest.mark.parametrize("scheme", ["picard", "full"])
def test_batch_matches_oracle_per_instance(lll, scheme):
    inst = _instances(6, 6 * 700)
    b, keep = lll.lll_batch_init(inst)
    try:
        lll.lll_batch_simulate(b, lll.SCHEMES[scheme], 42)
        got = _prices(lll, b, inst)
    finally:
        lll.lll_batch_destroy(b)
    code = ora.PICARD if scheme == "picard" else ora.FULL
    for q, (wl, x, W) in enumerate(inst):
        ref = ora.simulate(ora.OracleModel(wl, x, W), code, seed=42, inst=q)
        assert np.abs(got[q][0] - ref["price"]).max() <= 1e-7, (q, wl.N)


def test_graph_replay_and_launch_shapes(lll):
    inst = _instances(24, 1 << 16, seed=9)
    b, keep = lll.lll_batch_init(inst)
    try:
        lll.lll_batch_simulate(b, lll.LLL_PICARD, 7)
        eager = _prices(lll, b, inst)
        lll.lll_batch_use_graph(b, True)
        for _ in range(2):
            lll.lll_batch_simulate(b, lll.LLL_PICARD, 7)
            graph = _prices(lll, b, inst)
            for (pe, _), (pg, _) in zip(eager, graph):
                assert np.array_equal(pe, pg)
        lll.lll_batch_simulate(b, lll.LLL_PICARD, 8)  # new seed through the same graph
        other = _prices(lll, b, inst)
        assert any(not np.array_equal(pe, po) for (pe, _), (po, _) in zip(eager, other))
        lll.lll_batch_use_graph(b, False)
        lll.lll_batch_set_launch(b, 64, 1, 8)
        lll.lll_batch_simulate(b, lll.LLL_PICARD, 7)
        shaped = _prices(lll, b, inst)
        for (pe, _), (ps, _) in zip(eager, shaped):
            assert np.allclose(pe, ps, rtol=1e-12, atol=1e-18)
    finally:
        lll.lll_batch_destroy(b)


def test_claimed_items_run_every_tile_once(lll):
    """About 2^21 paths over 8 instances: many more tiles than resident blocks,
    so items span several tiles and every block claims many of them, in an
    order that changes from launch to launch.  Repeated launches give
    bit-identical prices; instance 0 (Philox word 1 = 0, as a single context
    draws) equals its own single-context simulation of the same paths, and
    every instance equals a launch with 64-thread tiles and one with two paths
    per thread (other tiles, other items), all within FP64 rounding of the
    grouping -- a tile run twice or not at all would move a price by about
    1/(tiles of the instance).  The Picard scheme runs between the full
    scheme's launches, each scheme on its own cached schedule."""
    inst = _instances(8, 1 << 21, seed=13)
    b, keep = lll.lll_batch_init(inst)
    try:
        runs = []
        for _ in range(3):
            lll.lll_batch_simulate(b, lll.LLL_FULL, 5)
            runs.append(_prices(lll, b, inst))
            lll.lll_batch_simulate(b, lll.LLL_PICARD, 5)  # the other scheme's schedule in between
        lll.lll_batch_set_launch(b, 64, 0, 0)
        lll.lll_batch_simulate(b, lll.LLL_FULL, 5)
        small = _prices(lll, b, inst)
        # two paths per thread (tiles of 256 paths): the same per-path arithmetic
        lll.lll_batch_set_launch(b, 128, 0, 16, 2, scheme="full")
        lll.lll_batch_simulate(b, lll.LLL_FULL, 5)
        pairs = _prices(lll, b, inst)
    finally:
        lll.lll_batch_destroy(b)
    for r in runs[1:]:
        for (p0, _), (p1, _) in zip(runs[0], r):
            assert np.array_equal(p0, p1)
    for q, ((p0, _), (ps, _), (pp, _)) in enumerate(zip(runs[0], small, pairs)):
        assert np.allclose(p0, ps, rtol=1e-12, atol=1e-18), q
        assert np.allclose(p0, pp, rtol=1e-12, atol=1e-18), q
    wl, x, W = inst[0]
    sim = lll.LevyLibor(wl, x, W)
    try:
        sim.set_launch(128, 0, 0, 1, 1)  # one lane per path: the batch kernel's arithmetic
        sim.simulate("full", seed=5)
        p, _ = sim.prices()
    finally:
        sim.close()
    assert np.allclose(runs[0][0][0], p, rtol=1e-12, atol=1e-18)


def test_launch_shape_validation(lll):
    """Out-of-range launch values are refused with LLL_EINVAL and leave the
    batch usable."""
    inst = _instances(2, 2 * 300, seed=3)
    b, keep = lll.lll_batch_init(inst)
    try:
        for args, kw in (((128, 0, 0, 3), {}), ((100, 0, 0, 1), {}), ((128, -1, 0, 1), {}),
                         ((128, 0, 0, 1), {"scheme": 5})):
            with pytest.raises(lll.LLLError) as e:
                lll.lll_batch_set_launch(b, *args, **kw)
            assert e.value.code == lll.LLL_EINVAL
        lll.lll_batch_simulate(b, lll.LLL_PICARD, 42)
        p, _ = lll.lll_batch_prices(b, 0, inst[0][0].n, inst[0][0].strikes.shape[1])
        assert np.all(np.isfinite(p))
    finally:
        lll.lll_batch_destroy(b)


def test_batch_with_96_nodes(lll):
    """Instances on a 96-node rule: one path per thread against the oracle;
    two paths per thread (compiled for up to 64 padded nodes) is refused with
    LLL_EUNSUPPORTED and leaves the batch usable."""
    import dataclasses

    inst = []
    for wl in workloads.batched_instances(n_inst=3, total_paths=3 * 400, seed=21):
        wl = dataclasses.replace(wl, Q=96, paths=max(wl.paths, 1))
        x, W = quadrature.rule_for(wl)
        inst.append((wl, x, W))
    b, keep = lll.lll_batch_init(inst)
    try:
        lll.lll_batch_set_launch(b, 128, 0, 0, 2, scheme="picard")
        with pytest.raises(lll.LLLError) as e:
            lll.lll_batch_simulate(b, lll.LLL_PICARD, 42)
        assert e.value.code == lll.LLL_EUNSUPPORTED
        lll.lll_batch_set_launch(b, 128, 0, 0, 1, scheme="picard")
        lll.lll_batch_simulate(b, lll.LLL_PICARD, 42)
        got = _prices(lll, b, inst)
    finally:
        lll.lll_batch_destroy(b)
    for q, (wl, x, W) in enumerate(inst):
        ref = ora.simulate(ora.OracleModel(wl, x, W), ora.PICARD, seed=42, inst=q)
        assert np.abs(got[q][0] - ref["price"]).max() <= 1e-7, (q, wl.N)
