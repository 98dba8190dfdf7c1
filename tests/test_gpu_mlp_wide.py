"""The learned compensator with the 256-wide vector head on the N = 120
workload (input (t, u_0 .. u_119) padded to 128, four hidden layers of 256,
119 outputs): LLL_MLP runs it as one persistent tcgen05 kernel
(lll_mlp_wide.cu) -- per 128-path tile, the network layer after layer with
the activations in shared memory and the weights streamed by TMA, the Euler
step and the payoffs.

Any network defines a scheme, so a seeded random network with a small output
unit s_y (the size of the learned part of the drift) is checked against the
FP64 oracle of the scheme with the same Philox increments.  Bound per
log-rate: T_N s_y 0.05 -- BF16 weights and activations give each output a
relative error of a few 2^-9, and the error of the drift integrates over at
most T_N years (the per-rate and N = 40 vector-head tests use the same bound).

* every path of three tiles (two full, one ragged: every TMEM lane quadrant,
  column quarter and CTA role) against the oracle, and the prices;
* at 152 x 2 x 128 + 77 paths, where every CTA runs two or three tiles in
  turn, sampled paths of second and third tiles (the ragged last one among
  them) against the oracle one by one, and the prices against the
  layer-by-layer path;
* failure detection without a GPU fault: with the MMA lane stalled, the
  bounded waits give up, the results read back as LLL_ETIMEOUT and the next
  simulation on the same context is bit for bit the reference;
* co-terminal swaptions against the swaption prices of the oracle's paths;
* the two- and three-layer instantiations with a one-K-block input (N = 10).
"""
import numpy as np
import pytest

from oracle import mlp as omlp
from oracle import oracle as ora
from oracle import quadrature
from paper_1006_3340_gb300 import workloads

pytestmark = pytest.mark.gpu
H, L = 256, 4
S_Y = 2e-4


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
def wide(lll):
    """long_dated with a seeded random 256 x 4 vector-head network."""
    wl = workloads.long_dated(paths=1 << 16)
    x, W = quadrature.rule_for(wl)
    sim = lll.LevyLibor(wl, x, W)
    lll.lll_mlp_init_head(sim.ctx, H, L, 1, seed=33)
    n_params, in_dim, in_pad, offs = lll.lll_mlp_layout(sim.ctx, L)
    head, outputs = lll.lll_mlp_shape(sim.ctx)
    assert (head, in_dim, in_pad, outputs) == (1, 121, 128, 128)
    flat, scales = lll.lll_mlp_params(sim.ctx, 0, count=n_params)
    scales = np.array(scales, dtype=np.float32)
    scales[4] = S_Y
    lll.lll_mlp_params(sim.ctx, 1, flat, scales=scales)
    params = omlp.params_from_flat(flat, offs, L, H, in_dim, in_pad, outputs=outputs)
    yield wl, x, W, sim, params, scales
    sim.close()


def _tol(wl, scales):
    return wl.N * wl.delta * float(scales[4]) * 0.05


TILE_PATHS = 2 * 128 + 37


def test_wide_vector_head_matches_fp64_scheme_path_by_path(lll, wide):
    wl, x, W, sim, params, scales = wide
    cnt = TILE_PATHS
    sim.simulate("mlp", paths=cnt, snapshots=cnt)
    z = sim.paths(0, cnt).astype(np.float64)
    p, _ = sim.prices()
    ref = omlp.simulate_scheme(ora.OracleModel(wl, x, W), params, scales, npaths=cnt, head=1)
    mask = ~np.isnan(ref["snap"])
    assert np.array_equal(mask, ~np.isnan(z))
    tol = _tol(wl, scales)
    d = np.abs(z - ref["snap"])
    per_path = np.nanmax(d.reshape(cnt, -1), axis=1)
    assert np.all(per_path <= tol), (np.argmax(per_path), per_path.max(), tol)
    assert np.median(per_path) <= 0.25 * tol, (np.median(per_path), tol)
    assert np.abs(p - ref["price"]).max() <= 1e-2 * tol


def test_wide_kernel_runs_by_default_and_layered_agrees(lll, wide):
    """The default kernel choice for this network is the persistent one (it is
    several times faster than the layer-by-layer path, which the bench records);
    both give the same prices to the BF16 bound of the scheme."""
    wl, x, W, sim, params, scales = wide
    cnt = 4096 + 77
    try:
        lll.lll_mlp_set_kernel(sim.ctx, "tc")
        sim.simulate("mlp", paths=cnt)
        p_w, _ = sim.prices()
        lll.lll_mlp_set_kernel(sim.ctx, "auto")
        sim.simulate("mlp", paths=cnt)
        p_a, _ = sim.prices()
        lll.lll_mlp_set_kernel(sim.ctx, "layered")
        sim.simulate("mlp", paths=cnt)
        p_l, _ = sim.prices()
    finally:
        lll.lll_mlp_set_kernel(sim.ctx, "auto")
    assert np.array_equal(p_w, p_a)
    assert np.abs(p_w - p_l).max() <= 1e-2 * _tol(wl, scales)


# every CTA (152 on a GB300) runs two tiles, the first 77 paths' CTA a third
MULTI_PATHS = 152 * 2 * 128 + 77
STRIDE = 9731  # samples 0, 9731, 19462, 29193, 38924: first, second and third (ragged) tiles


def test_wide_kernel_sampled_paths_of_later_tiles_match_fp64(lll, wide):
    wl, x, W, sim, params, scales = wide
    cnt = MULTI_PATHS
    samples = np.arange(0, cnt, STRIDE)
    assert samples[-1] >= cnt - 77  # the ragged last tile is sampled
    sim.simulate("mlp", paths=cnt, snapshots=len(samples), snapshot_stride=STRIDE)
    z = sim.paths(0, len(samples)).astype(np.float64)
    p_w, _ = sim.prices()
    model = ora.OracleModel(wl, x, W)
    tol = _tol(wl, scales)
    for i, lp in enumerate(samples):
        ref = omlp.simulate_scheme(model, params, scales, path0=int(lp), npaths=1, head=1)
        mask = ~np.isnan(ref["snap"][0])
        assert np.array_equal(mask, ~np.isnan(z[i]))
        err = np.abs(z[i][mask] - ref["snap"][0][mask]).max()
        assert err <= tol, (int(lp), err, tol)
    try:
        lll.lll_mlp_set_kernel(sim.ctx, "layered")
        sim.simulate("mlp", paths=cnt)
        p_l, _ = sim.prices()
    finally:
        lll.lll_mlp_set_kernel(sim.ctx, "auto")
    assert np.abs(p_w - p_l).max() <= 1e-2 * tol


def test_wide_kernel_bounded_waits_give_up_and_context_stays_usable(lll, wide):
    wl, x, W, sim, params, scales = wide
    cnt = 2048
    sim.simulate("mlp", paths=cnt)
    ref, _ = sim.prices()
    lll.lll_inject(sim.ctx, lll.LLL_INJECT_MMA_STALL)
    sim.simulate("mlp", paths=cnt)
    with pytest.raises(lll.LLLError) as e:
        sim.prices()
    assert e.value.code == -4
    sim.simulate("mlp", paths=cnt)
    again, _ = sim.prices()
    assert np.array_equal(ref, again)


def test_wide_kernel_swaptions_match_fp64_scheme(lll, wide):
    """Co-terminal payer swaptions on the same fused kernel (the pricing warps
    form P and S from the shared state in rate order), against the swaption
    prices of the FP64 oracle's own paths of the scheme.  Bound: each path's
    log-rates are within T_N s_y 0.05 of the oracle's (previous tests), and a
    swaption payoff moves by at most (1 + delta L_m) P + K delta S ~ 3 per unit
    log-rate change summed over the rates, so prices agree within 3 T_N s_y 0.05
    times the median path error fraction (0.25, see the path test)."""
    wl, x, W, sim, params, scales = wide
    cnt = TILE_PATHS
    try:
        sim.set_product("swaption")
        sim.simulate("mlp", paths=cnt)
        p, _ = sim.prices()
        lll.lll_mlp_set_kernel(sim.ctx, "layered")
        sim.simulate("mlp", paths=cnt)
        p_l, _ = sim.prices()
    finally:
        lll.lll_mlp_set_kernel(sim.ctx, "auto")
        sim.set_product("caplet")
    ref = omlp.simulate_scheme(ora.OracleModel(wl, x, W), params, scales, npaths=cnt, head=1)
    want = ora.swaption_prices(wl, ref["snap"], wl.strikes)
    tol = 3.0 * 0.25 * _tol(wl, scales)
    assert np.abs(p - want).max() <= tol, (np.abs(p - want).max(), tol)
    assert np.abs(p - p_l).max() <= tol


@pytest.mark.parametrize("layers", [2, 3])
def test_wide_kernel_small_network_variants_match_fp64(lll, layers):
    """The other instantiations of the fused kernel: two and three hidden
    layers of 256 and an input of one 64-wide K block (N = 10: input 11 padded
    to 16), over two full tiles and a ragged third, path by path against the
    FP64 oracle (same bound as above)."""
    wl = workloads.small_plain(paths=2 * 128 + 37)
    x, W = quadrature.rule_for(wl)
    sim = lll.LevyLibor(wl, x, W)
    try:
        lll.lll_mlp_init_head(sim.ctx, H, layers, 1, seed=11 + layers)
        n_params, in_dim, in_pad, offs = lll.lll_mlp_layout(sim.ctx, layers)
        head, outputs = lll.lll_mlp_shape(sim.ctx)
        assert in_pad <= 64
        flat, scales = lll.lll_mlp_params(sim.ctx, 0, count=n_params)
        scales = np.array(scales, dtype=np.float32)
        scales[4] = 1e-3
        lll.lll_mlp_params(sim.ctx, 1, flat, scales=scales)
        cnt = wl.paths
        sim.simulate("mlp", paths=cnt, snapshots=cnt)
        z = sim.paths(0, cnt).astype(np.float64)
        p, _ = sim.prices()
    finally:
        sim.close()
    params = omlp.params_from_flat(flat, offs, layers, H, in_dim, in_pad, outputs=outputs)
    ref = omlp.simulate_scheme(ora.OracleModel(wl, x, W), params, scales, npaths=cnt, head=1)
    mask = ~np.isnan(ref["snap"])
    assert np.array_equal(mask, ~np.isnan(z))
    tol = _tol(wl, scales)
    per_path = np.nanmax(np.abs(z - ref["snap"]).reshape(cnt, -1), axis=1)
    assert np.all(per_path <= tol), (per_path.max(), tol)
    assert np.abs(p - ref["price"]).max() <= 1e-2 * tol
