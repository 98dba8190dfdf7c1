"""Vector-head learned compensator (lll_mlp_cfg.head = 1): one evaluation per
(path, Euler step) gives every rate's compensator.

* GPU output and gradients against the FP64 oracle (masked MSE over the first
  n output columns), BF16 tolerances as for the per-rate network.
* The trained network prices within 0.5 bp of the quadrature full scheme and
  improves the pathwise log-rates over the scheme without the learned part.
* Path by path against the FP64 oracle of the same scheme (same network,
  same Philox increments), with the BF16 bound T_N s_y 0.05 on log-rates.
"""
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


@pytest.mark.parametrize("gemm", ["tc", "mma_sync"])
def test_vector_head_forward_and_gradients_match_fp64(lll, gemm):
    wl = workloads.large_single(paths=1024)
    sim = lll.LevyLibor(wl)
    lll.lll_set_gemm_kernel(gemm)
    try:
        lll.lll_mlp_init(sim.ctx, H, L, seed=5, head=1)
        head, O = lll.lll_mlp_shape(sim.ctx)
        assert (head, O) == (1, 48)
        n_params, in_dim, in_pad, offs = lll.lll_mlp_layout(sim.ctx, L)
        assert in_dim == 1 + wl.N
        flat, _ = lll.lll_mlp_params(sim.ctx, 0, count=n_params)
        rng = np.random.default_rng(6)
        rows = 512
        x = omlp.bf16_round(rng.normal(size=(rows, in_dim)))
        y = rng.normal(size=(rows, O)).astype(np.float32)
        out, g, loss = lll.lll_mlp_eval(sim.ctx, x, y, n_params, want_grads=True)
    finally:
        lll.lll_set_gemm_kernel("tc")
        sim.close()
    params = omlp.params_from_flat(flat, offs, L, H, in_dim, in_pad, outputs=O)
    out_o = omlp.forward_vec(params, x.astype(np.float64))
    loss_o, grads_o = omlp.loss_and_grads_vec(params, x.astype(np.float64), y.astype(np.float64), wl.n)
    assert np.abs(out - out_o).max() <= 2e-2 * np.abs(out_o).max()
    assert abs(loss - loss_o) <= 2e-2 * loss_o
    for l in range(L + 1):
        off_w, off_b = offs[2 * l], offs[2 * l + 1]
        din = in_pad if l == 0 else H
        rows_w = O if l == L else H
        gW = g[off_w: off_w + rows_w * din].reshape(rows_w, din)
        gW = gW[:, :in_dim] if l == 0 else gW
        gb = g[off_b: off_b + rows_w]
        oW, ob = grads_o[l]
        assert np.linalg.norm(gW - oW) <= 3e-2 * np.linalg.norm(oW), l
        assert np.linalg.norm(gb - ob) <= 3e-2 * np.linalg.norm(ob) + 1e-12, l


@pytest.fixture(scope="module")
def trained_vec(lll):
    wl = workloads.large_single(paths=1 << 16)
    x, W = quadrature.rule_for(wl)
    sim = lll.LevyLibor(wl, x, W)
    loss = lll.lll_mlp_train(sim.ctx, hidden=H, layers=L, train_paths=1 << 16, records_per_path=8,
                             epochs=40, batch=4096, lr=2e-3, lr_final=1e-4, seed=7, head=1)
    yield wl, x, W, sim, loss
    sim.close()


def _run(sim, scheme, count):
    sim.simulate(scheme, snapshots=count)
    p, se = sim.prices()
    return p, se, sim.paths(0, count).astype(np.float64)


def test_vector_head_within_half_bp_and_gains(lll, trained_vec):
    wl, x, W, sim, loss = trained_vec
    cnt = 4096
    p_full, _, z_full = _run(sim, "full", cnt)
    p_vec, _, z_vec = _run(sim, "mlp", cnt)
    assert np.abs(p_vec - p_full).max() <= 5e-5, np.abs(p_vec - p_full).max()
    n_params, _, _, _ = lll.lll_mlp_layout(sim.ctx, L)
    flat, scales = lll.lll_mlp_params(sim.ctx, 0, count=n_params)
    try:
        lll.lll_mlp_params(sim.ctx, 1, np.zeros_like(flat), scales=scales)  # learned part removed
        p_zero, _, z_zero = _run(sim, "mlp", cnt)
    finally:
        lll.lll_mlp_params(sim.ctx, 1, flat, scales=scales)
    mask = ~np.isnan(z_full)
    err_vec = np.abs(z_vec[mask] - z_full[mask]).max()
    err_zero = np.abs(z_zero[mask] - z_full[mask]).max()
    assert err_vec < 0.5 * err_zero, (err_vec, err_zero)


@pytest.fixture(scope="module")
def fp64_vec(lll, trained_vec):
    wl, x, W, sim, loss = trained_vec
    n_params, in_dim, in_pad, offs = lll.lll_mlp_layout(sim.ctx, L)
    flat, scales = lll.lll_mlp_params(sim.ctx, 0, count=n_params)
    _, O = lll.lll_mlp_shape(sim.ctx)
    params = omlp.params_from_flat(flat, offs, L, H, in_dim, in_pad, outputs=O)
    return scales, omlp.simulate_scheme(ora.OracleModel(wl, x, W), params, scales, npaths=ORACLE_PATHS,
                                        head=1)


# Two CTAs of the tensor-memory kernel (both 128-row tiles, every TMEM lane
# quadrant and column quarter) and a ragged 37-path third.
ORACLE_PATHS = 2 * 256 + 37


@pytest.mark.parametrize("kind", ["tc", "layered"])
def test_vector_head_matches_fp64_scheme_path_by_path(lll, trained_vec, fp64_vec, kind):
    """Path by path against the FP64 oracle of the vector-head scheme over
    every tile, lane quadrant and column quarter of two CTAs and a ragged
    third; bound T_N s_y 0.05 on each log-rate (see the per-rate test)."""
    wl, x, W, sim, loss = trained_vec
    cnt = ORACLE_PATHS
    scales, ref = fp64_vec
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
    assert d[mask].max() <= tol, (d[mask].max(), tol)
    per_path = np.nanmax(d.reshape(cnt, -1), axis=1)
    assert np.all(per_path <= tol), np.argmax(per_path)
    assert np.median(per_path) <= 0.25 * tol, (np.median(per_path), tol)
    assert np.abs(p - ref["price"]).max() <= 1e-2 * tol


def test_tcgen05_and_layered_vector_head_agree(lll, trained_vec):
    """Same network, same paths: the fused tensor-memory kernel and the
    layer-by-layer path differ only in FP32 accumulation order (2e-6 in
    log-rate, 1e-9 in price, ragged path counts included)."""
    wl, x, W, sim, loss = trained_vec
    cnt = 4096
    try:
        lll.lll_mlp_set_kernel(sim.ctx, "tc")
        p_t, _, z_t = _run(sim, "mlp", cnt)
        sim.simulate("mlp", paths=wl.paths - 77)
        p_tr, _ = sim.prices()
        lll.lll_mlp_set_kernel(sim.ctx, "layered")
        p_l, _, z_l = _run(sim, "mlp", cnt)
        sim.simulate("mlp", paths=wl.paths - 77)
        p_lr, _ = sim.prices()
        lll.lll_mlp_set_kernel(sim.ctx, "warp")  # the mma.sync kernel has no vector head
        with pytest.raises(lll.LLLError):
            sim.simulate("mlp", paths=256)
    finally:
        lll.lll_mlp_set_kernel(sim.ctx, "auto")
    mask = ~np.isnan(z_t)
    assert np.abs(z_t[mask] - z_l[mask]).max() <= 2e-6
    assert np.abs(p_t - p_l).max() <= 1e-9
    assert np.abs(p_tr - p_lr).max() <= 1e-9


def test_vector_head_bounded_waits_give_up_and_context_stays_usable(lll, trained_vec):
    """Failure detection of the vector-head kernel without a GPU fault: with
    LLL_INJECT_MMA_STALL its MMA lane issues nothing, so every bounded wait
    runs out. Those are the product waits and the increment and maturity
    barriers between column quarters. The launch ends by itself, the results
    read back as LLL_ETIMEOUT (-4), and the next simulation on the same context
    reproduces the reference prices bit for bit."""
    wl, x, W, sim, loss = trained_vec
    cnt = 4096
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
