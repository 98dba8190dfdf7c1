"""The learned compensator on the GPU (BF16 tensor-core kernels) against the
FP64 oracle MLP, and the LLL_MLP scheme against the quadrature full scheme.

Tolerances follow from BF16: weights, inputs and hidden activations are
rounded to 8 significant bits (relative 2^-9), accumulation is FP32, so the
network output and every gradient tensor must agree with the FP64 oracle
evaluated on the same BF16-rounded weights and inputs to a few 1e-2 in
relative norm.  The scheme must price caplets within 0.5 bp (5e-5) of the
quadrature full scheme; the gain test compares it with the same scheme with
the learned part removed (a zero network, i.e. the compensator at zero
weights C_i only).
"""
import os
import tempfile

import numpy as np
import pytest

from oracle import mlp as omlp
from oracle import oracle as ora
from oracle import quadrature
from paper_1006_3340_gb300 import workloads

pytestmark = pytest.mark.gpu
H, L = 128, 3


@pytest.fixture(scope="module")
def lll():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1006_3340_gb300 import lll as mod

    mod.load()
    return mod


def bf16(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _oracle_params(flat, offs, in_dim, in_pad):
    params = []
    for l in range(L):
        din = in_pad if l == 0 else H
        W = bf16(flat[offs[2 * l]: offs[2 * l] + H * din]).reshape(H, din).astype(np.float64)
        if l == 0:
            W = W[:, :in_dim]
        params.append((W, flat[offs[2 * l + 1]: offs[2 * l + 1] + H].astype(np.float64)))
    wout = bf16(flat[offs[2 * L]: offs[2 * L] + H]).astype(np.float64)[None, :]
    params.append((wout, flat[offs[2 * L + 1]: offs[2 * L + 1] + 1].astype(np.float64)))
    return params


def _flat_grads(g, offs, in_dim, in_pad):
    out = []
    for l in range(L):
        din = in_pad if l == 0 else H
        W = g[offs[2 * l]: offs[2 * l] + H * din].reshape(H, din)
        if l == 0:
            assert np.all(W[:, in_dim:] == 0)
            W = W[:, :in_dim]
        out.append((W, g[offs[2 * l + 1]: offs[2 * l + 1] + H]))
    out.append((g[offs[2 * L]: offs[2 * L] + H][None, :], g[offs[2 * L + 1]: offs[2 * L + 1] + 1]))
    return out


@pytest.mark.parametrize("gemm", ["tc", "mma_sync"])
def test_forward_and_gradients_match_fp64_oracle(lll, gemm):
    """Forward output, loss and every gradient tensor of the GPU training pass
    (GEMMs on the tcgen05 kernel, the default, or the mma.sync kernel) against
    the FP64 oracle on the same BF16 weights and inputs."""
    wl = workloads.large_single(paths=1024)
    sim = lll.LevyLibor(wl)
    lll.lll_set_gemm_kernel(gemm)
    try:
        lll.lll_mlp_init(sim.ctx, H, L, seed=3)
        n_params, in_dim, in_pad, offs = lll.lll_mlp_layout(sim.ctx, L)
        flat, _ = lll.lll_mlp_params(sim.ctx, 0, count=n_params)
        rng = np.random.default_rng(5)
        rows = 1000
        x = bf16(rng.normal(size=(rows, in_dim)))
        y = rng.normal(size=rows).astype(np.float32)
        out, g, loss = lll.lll_mlp_eval(sim.ctx, x, y, n_params, want_grads=True)
    finally:
        lll.lll_set_gemm_kernel("tc")
        sim.close()
    params = _oracle_params(flat, offs, in_dim, in_pad)
    out_o, _ = omlp.forward(params, x.astype(np.float64))
    loss_o, grads_o = omlp.loss_and_grads(params, x.astype(np.float64), y.astype(np.float64))
    assert np.abs(out - out_o).max() <= 2e-2 * np.abs(out_o).max()
    assert abs(loss - loss_o) <= 2e-2 * loss_o
    for (gW, gb), (oW, ob) in zip(_flat_grads(g, offs, in_dim, in_pad), grads_o):
        assert np.linalg.norm(gW - oW) <= 3e-2 * np.linalg.norm(oW)
        assert np.linalg.norm(gb - ob) <= 3e-2 * np.linalg.norm(ob)


def test_training_reduces_loss_and_roundtrips_through_file(lll):
    wl = workloads.large_single(paths=4096)
    sim = lll.LevyLibor(wl)
    sim2 = lll.LevyLibor(wl)
    try:
        loss = lll.lll_mlp_train(sim.ctx, hidden=H, layers=L, train_paths=1 << 14, records_per_path=4,
                                 epochs=3, batch=4096, lr=2e-3, lr_final=2e-4, seed=11)
        assert loss < 0.1, loss  # targets are scaled to unit RMS
        n_params, in_dim, _, _ = lll.lll_mlp_layout(sim.ctx, L)
        x = bf16(np.random.default_rng(1).normal(size=(64, in_dim)) * 0.3)
        a, _, _ = lll.lll_mlp_eval(sim.ctx, x)
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "net.bin")
            lll.lll_mlp_save(sim.ctx, path)
            lll.lll_mlp_load(sim2.ctx, path)
        b, _, _ = lll.lll_mlp_eval(sim2.ctx, x)
        assert np.array_equal(a, b)
    finally:
        sim.close()
        sim2.close()


@pytest.fixture(scope="module")
def trained(lll):
    wl = workloads.large_single(paths=1 << 16)
    x, W = quadrature.rule_for(wl)
    sim = lll.LevyLibor(wl, x, W)
    loss = lll.lll_mlp_train(sim.ctx, hidden=H, layers=L, train_paths=1 << 16, records_per_path=8,
                             epochs=4, batch=8192, lr=2e-3, lr_final=1e-4, seed=7)
    yield wl, x, W, sim, loss
    sim.close()


def _run(sim, scheme, count):
    sim.simulate(scheme, snapshots=count)
    p, se = sim.prices()
    return p, se, sim.paths(0, count).astype(np.float64)


def test_mlp_scheme_within_half_bp_of_quadrature_and_gains_over_no_network(lll, trained):
    wl, x, W, sim, loss = trained
    cnt = 4096
    p_full, se_full, z_full = _run(sim, "full", cnt)
    p_mlp, _, z_mlp = _run(sim, "mlp", cnt)
    assert np.abs(p_mlp - p_full).max() <= 5e-5
    n_params, _, _, _ = lll.lll_mlp_layout(sim.ctx, L)
    flat, scales = lll.lll_mlp_params(sim.ctx, 0, count=n_params)
    try:
        lll.lll_mlp_params(sim.ctx, 1, np.zeros_like(flat), scales=scales)  # learned part removed
        p_zero, _, z_zero = _run(sim, "mlp", cnt)
    finally:
        lll.lll_mlp_params(sim.ctx, 1, flat, scales=scales)
    mask = ~np.isnan(z_full)
    err_mlp = np.abs(z_mlp[mask] - z_full[mask]).max()
    err_zero = np.abs(z_zero[mask] - z_full[mask]).max()
    assert err_mlp < 0.2 * err_zero, (err_mlp, err_zero)
    assert np.abs(p_mlp - p_full).max() <= np.abs(p_zero - p_full).max() + 1e-12


def test_mlp_scheme_against_fp64_oracle(lll, trained):
    wl, x, W, sim, loss = trained
    cnt = 2048
    sim.simulate("mlp", paths=cnt)
    p_mlp, _ = sim.prices()
    ref = ora.simulate(ora.OracleModel(wl, x, W), ora.FULL, npaths=cnt)
    assert np.abs(p_mlp - ref["price"]).max() <= 5e-5  # 0.5 bp of notional


def test_tcgen05_kernel_matches_mma_sync_kernel(lll, trained):
    """The tensor-memory kernel and the warp-level kernel evaluate the same
    network on the same paths: BF16 activations, FP32 accumulation in a
    different order (the tensor-memory kernel adds the rate's own inputs
    t, i, lambda_i to the first layer through a per-rate bias).  A rounding
    difference moves one activation by at most 2^-8 relative, which moves a
    drift by a small fraction of s_y; over the 312 steps the log-rates then
    agree to 2e-6.  A log-rate difference eps moves a caplet payoff by at most
    delta B(0,T_N) L (1 + delta L)^n eps < 1e-2 eps, so the prices agree to 2e-8."""
    wl, x, W, sim, loss = trained
    cnt = 4096
    try:
        lll.lll_mlp_set_kernel(sim.ctx, "warp")
        p_w, _, z_w = _run(sim, "mlp", cnt)
        lll.lll_mlp_set_kernel(sim.ctx, "tc")
        p_t, _, z_t = _run(sim, "mlp", cnt)
        sim.simulate("mlp", paths=wl.paths)  # full launch shape, ragged-free 2^16 paths
        lll.lll_mlp_set_kernel(sim.ctx, "warp")
        sim.simulate("mlp", paths=wl.paths - 77)  # ragged last tile
        p_wr, _ = sim.prices()
        lll.lll_mlp_set_kernel(sim.ctx, "tc")
        sim.simulate("mlp", paths=wl.paths - 77)
        p_tr, _ = sim.prices()
    finally:
        lll.lll_mlp_set_kernel(sim.ctx, "auto")
    mask = ~np.isnan(z_w)
    assert np.abs(z_t[mask] - z_w[mask]).max() <= 2e-6
    assert np.abs(p_t - p_w).max() <= 2e-8
    assert np.abs(p_tr - p_wr).max() <= 2e-8


# Paths compared with the FP64 oracle one by one: two CTAs of the tensor-
# memory kernel (two 128-row tiles each, all four TMEM lane quadrants and
# every epilogue warp) and a third CTA with a ragged 37-path tile; for the
# mma.sync kernel 17 warps of 32 paths and a ragged one.
ORACLE_PATHS = 2 * 256 + 37


@pytest.fixture(scope="module")
def fp64_scheme(lll, trained):
    """The FP64 oracle of the scheme with the trained network, first ORACLE_PATHS paths."""
    wl, x, W, sim, loss = trained
    n_params, in_dim, in_pad, offs = lll.lll_mlp_layout(sim.ctx, L)
    flat, scales = lll.lll_mlp_params(sim.ctx, 0, count=n_params)
    params = omlp.params_from_flat(flat, offs, L, H, in_dim, in_pad)
    return scales, omlp.simulate_scheme(ora.OracleModel(wl, x, W), params, scales, npaths=ORACLE_PATHS)


@pytest.mark.parametrize("kind", ["tc", "warp", "layered"])
def test_mlp_kernels_match_fp64_scheme_path_by_path(lll, trained, fp64_scheme, kind):
    """Every LLL_MLP kernel against the FP64 oracle of the same scheme with the
    same (BF16-stored) network, on identical Philox increments, path by path
    over both tiles of two CTAs and a ragged third.  The GPU feeds BF16
    features and activations through the network, so one evaluation of f may
    differ from the FP64 one by a few per cent of its unit RMS (the forward
    test's bound, 2e-2 of max |f|, plus the SiLU approximation); a log-rate
    offset integrates h s_y times that over at most T_N / h steps:
    |d log L| <= T_N s_y 0.05.  The median error must sit far below that
    bound (rounding errors of single evaluations do not add up coherently)."""
    wl, x, W, sim, loss = trained
    cnt = ORACLE_PATHS
    scales, ref = fp64_scheme
    try:
        lll.lll_mlp_set_kernel(sim.ctx, kind)
        sim.simulate("mlp", paths=cnt, snapshots=cnt)
        z = sim.paths(0, cnt).astype(np.float64)
        p, _ = sim.prices()
    finally:
        lll.lll_mlp_set_kernel(sim.ctx, "auto")
    mask = ~np.isnan(ref["snap"])
    assert np.array_equal(mask, ~np.isnan(z))
    tol = wl.N * wl.delta * float(scales[4]) * 0.05
    d = np.abs(z - ref["snap"])
    err = d[mask].max()
    assert err <= tol, (err, tol)
    # every path, tile and lane quadrant meets the bound (not only the worst)
    per_path = np.nanmax(d.reshape(cnt, -1), axis=1)
    assert np.all(per_path <= tol), np.argmax(per_path)
    assert np.median(per_path) <= 0.25 * tol, (np.median(per_path), tol)
    # payoff sensitivity to a log-rate: delta B(0,T_N) L (1 + delta L)^n < 1e-2
    assert np.abs(p - ref["price"]).max() <= 1e-2 * tol


def test_layered_path_matches_fused_kernel(lll, trained):
    """The layer-by-layer path (training GEMMs over all rows of a step) and the
    fused tensor-memory kernel evaluate the same network on the same paths."""
    wl, x, W, sim, loss = trained
    cnt = 4096
    try:
        lll.lll_mlp_set_kernel(sim.ctx, "tc")
        p_t, _, z_t = _run(sim, "mlp", cnt)
        lll.lll_mlp_set_kernel(sim.ctx, "layered")
        p_l, _, z_l = _run(sim, "mlp", cnt)
        sim.simulate("mlp", paths=wl.paths - 77)  # several chunks' worth of rows, ragged end
        p_lr, _ = sim.prices()
        lll.lll_mlp_set_kernel(sim.ctx, "tc")
        sim.simulate("mlp", paths=wl.paths - 77)
        p_tr, _ = sim.prices()
    finally:
        lll.lll_mlp_set_kernel(sim.ctx, "auto")
    mask = ~np.isnan(z_t)
    assert np.abs(z_l[mask] - z_t[mask]).max() <= 2e-6
    assert np.abs(p_l - p_t).max() <= 2e-8  # bound of the test above
    assert np.abs(p_lr - p_tr).max() <= 2e-8


def test_wide_network_on_long_dated_workload_matches_fp64_scheme(lll):
    """The N=120 workload with the 123 -> 4 x 256 -> 1 network (no fused kernel
    holds it: LLL_MLP runs layer by layer).  Any network defines a scheme, so
    a seeded random one with a small output unit s_y is checked path by path
    against the FP64 oracle of the scheme."""
    wl = workloads.long_dated(paths=2)
    x, W = quadrature.rule_for(wl)
    sim = lll.LevyLibor(wl, x, W)
    try:
        lll.lll_mlp_init(sim.ctx, 256, 4, seed=21)
        n_params, in_dim, in_pad, offs = lll.lll_mlp_layout(sim.ctx, 4)
        assert (in_dim, in_pad) == (123, 128)
        flat, scales = lll.lll_mlp_params(sim.ctx, 0, count=n_params)
        scales = np.array(scales, dtype=np.float32)
        scales[4] = 2e-4  # s_y: drift perturbation of the order of the learned part
        lll.lll_mlp_params(sim.ctx, 1, flat, scales=scales)
        sim.simulate("mlp", paths=wl.paths, snapshots=wl.paths)
        z = sim.paths(0, wl.paths).astype(np.float64)
        p, _ = sim.prices()
    finally:
        sim.close()
    params = omlp.params_from_flat(flat, offs, 4, 256, in_dim, in_pad)
    ref = omlp.simulate_scheme(ora.OracleModel(wl, x, W), params, scales, npaths=wl.paths)
    mask = ~np.isnan(ref["snap"])
    assert np.array_equal(mask, ~np.isnan(z))
    tol = wl.N * wl.delta * float(scales[4]) * 0.05
    err = np.abs(z[mask] - ref["snap"][mask]).max()
    assert err <= tol, (err, tol)
    assert np.abs(p - ref["price"]).max() <= 1e-2 * tol


def test_bounded_wait_gives_up_and_context_stays_usable(lll, trained):
    """Failure detection without a GPU fault: with LLL_INJECT_MMA_STALL the
    MMA warp issues nothing, the epilogue's bounded waits run out, the launch
    ends by itself and the results read back as LLL_ETIMEOUT (-4); the next
    simulation on the same context is exact again."""
    wl, x, W, sim, loss = trained
    cnt = 2048
    try:
        lll.lll_mlp_set_kernel(sim.ctx, "tc")
        sim.simulate("mlp", paths=cnt)
        ref, _ = sim.prices()
        lll.lll_inject(sim.ctx, lll.LLL_INJECT_MMA_STALL)
        sim.simulate("mlp", paths=cnt)
        with pytest.raises(lll.LLLError) as e:
            sim.prices()
        assert e.value.code == -4
        sim.simulate("mlp", paths=cnt)
        again, _ = sim.prices()
    finally:
        lll.lll_mlp_set_kernel(sim.ctx, "auto")
    assert np.array_equal(ref, again)
