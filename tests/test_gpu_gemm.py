"""The learned compensator's GEMM kernels (lll_gemm_bf16 through the C ABI):
the tcgen05 kernel (tensor memory accumulator, swizzled shared-memory
operands) and the mma.sync kernel, against an FP64 numpy product of the same
BF16 operands.

Bound: FP32 accumulation of K products of BF16 values, |error| <= K 2^-23
sum_k |a_k b_k| per element (a loose form of the standard summation bound),
checked as 2e-5 of the row's sum of |a b| plus a tiny absolute term.  The
epilogues' SiLU uses tanh.approx (about 2^-11 relative error) and rounds to
BF16 (2^-9), so H agrees to 4e-3 relative to max(|z|, 1).

Shapes cover every operand layout the training and inference passes use,
ragged M, N and K (partial tiles, partial 8-element chunks), leading
dimensions that are not multiples of 8 (the kernel's scalar staging path),
two N tiles, and split-K with uneven ranges.
"""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lll():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1006_3340_gb300 import lll as mod

    mod.load()
    yield mod
    mod.lll_set_gemm_kernel("tc")


def _bf16(rng, shape, scale=1.0):
    v = omlp.bf16_round(rng.normal(size=shape) * scale)
    return v, (v.view(np.uint32) >> 16).astype(np.uint16)


def _silu(z):
    return z / (1.0 + np.exp(-z))


def _silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _bits_to_f(h):
    return (h.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


CASES = [
    # ta, tb, epi, M, N, K, lda_pad, ldb_pad, splits
    (0, 1, 1, 300, 200, 75, 0, 0, 1),     # forward layer: ragged everything, lda = K = 75 (scalar staging)
    (0, 1, 1, 256, 128, 48, 0, 0, 1),     # the N=40 per-rate first layer (in_pad 48)
    (0, 1, 1, 1000, 256, 256, 0, 0, 1),   # a 256-wide hidden layer (one 256-column tile)
    (0, 1, 1, 200, 300, 128, 8, 8, 1),    # two N tiles of 256, padded leading dimensions
    (0, 1, 0, 1000, 128, 256, 0, 0, 1),   # vector-head output layer (FP32 out)
    (0, 1, 0, 77, 48, 128, 0, 0, 1),
    (0, 0, 2, 257, 129, 64, 0, 0, 1),     # backward dX with SiLU'
    (0, 0, 2, 300, 256, 256, 0, 0, 1),
    (0, 1, 2, 333, 128, 128, 0, 0, 1),    # dX from the transposed weight copy (tcgen05)
    (1, 0, 0, 128, 48, 1000, 0, 0, 4),    # dW = dZ^T H, split-K (uneven ranges)
    (1, 0, 0, 256, 123, 8192, 0, 5, 16),  # dW of a first layer, odd ldb
    (0, 0, 0, 100, 70, 90, 3, 0, 2),      # plain product, odd lda, split-K
]


@pytest.mark.parametrize("kind", ["tc", "mma_sync"])
@pytest.mark.parametrize("case", CASES, ids=[f"t{c[0]}{c[1]}e{c[2]}_{c[3]}x{c[4]}x{c[5]}" for c in CASES])
def test_gemm_matches_fp64_product(lll, kind, case):
    ta, tb, epi, M, N, K, pa, pb, splits = case
    rng = np.random.default_rng(M * 7 + N * 13 + K)
    lda = (M if ta else K) + pa
    ldb = (K if tb else N) + pb
    Af, Ab = _bf16(rng, ((K if ta else M), lda))
    Bf, Bb = _bf16(rng, ((N if tb else K), ldb), 0.1)
    A = (Af[:K, :M].T if ta else Af[:M, :K]).astype(np.float64)
    B = (Bf[:N, :K].T if tb else Bf[:K, :N]).astype(np.float64)
    ref = A @ B
    mag = np.abs(A) @ np.abs(B)
    tol = 2e-5 * mag + 1e-30
    bias = rng.normal(size=N).astype(np.float32) if epi == 1 else None
    Zin = rng.normal(size=(M, N)).astype(np.float32) if epi == 2 else None
    if kind == "mma_sync" and epi == 2 and tb == 1:
        pytest.skip("the mma.sync kernel reads dX's weights column-wise (tb = 0) only")
    lll.lll_set_gemm_kernel(kind)
    C, H = lll.lll_gemm_bf16(ta, tb, epi, Ab, lda, Bb, ldb, M, N, K, splits, bias, Zin)
    if epi == 0:
        assert np.all(np.abs(C - ref) <= tol), np.max(np.abs(C - ref) / (mag + 1e-30))
    elif epi == 1:
        z = ref + bias.astype(np.float64)
        assert np.all(np.abs(C - z) <= tol)
        h = _bits_to_f(H)
        assert np.all(np.abs(h - _silu(z)) <= 4e-3 * np.maximum(np.abs(z), 1.0)), np.max(np.abs(h - _silu(z)))
    else:
        d = ref * _silu_grad(Zin.astype(np.float64))
        assert np.all(np.abs(C - d) <= tol * 1.2 + 4e-3 * np.abs(d))
        h = _bits_to_f(H)
        assert np.all(np.abs(h - C) <= 2 ** -8 * np.abs(C) + 1e-30)


def test_tcgen05_and_mma_sync_agree(lll):
    """Both kernels on one forward layer: FP32 sums of the same BF16 products
    in different orders, so z agrees to the accumulation bound."""
    rng = np.random.default_rng(3)
    M, N, K = 4096, 128, 128
    _, Ab = _bf16(rng, (M, K))
    _, Bb = _bf16(rng, (N, K), 0.1)
    bias = rng.normal(size=N).astype(np.float32)
    lll.lll_set_gemm_kernel("tc")
    Ct, _ = lll.lll_gemm_bf16(0, 1, 1, Ab, K, Bb, K, M, N, K, 1, bias)
    lll.lll_set_gemm_kernel("mma_sync")
    Cm, _ = lll.lll_gemm_bf16(0, 1, 1, Ab, K, Bb, K, M, N, K, 1, bias)
    lll.lll_set_gemm_kernel("tc")
    assert np.max(np.abs(Ct - Cm)) <= 1e-4 * np.max(np.abs(Cm))


@pytest.mark.parametrize("epi,M,N,K", [(3, 300, 130, 256), (4, 128, 1000, 256), (4, 48, 333, 128)])
def test_bias_epilogues(lll, epi, M, N, K):
    """Epilogue 3 adds a bias per column, 4 per row (the vector head's output
    layer computed transposed, out^T = W_out H^T + b_out)."""
    rng = np.random.default_rng(epi * 100 + M)
    Af, Ab = _bf16(rng, (M, K))
    Bf, Bb = _bf16(rng, (N, K), 0.1)
    bias = rng.normal(size=(N if epi == 3 else M)).astype(np.float32)
    lll.lll_set_gemm_kernel("tc")
    C, _ = lll.lll_gemm_bf16(0, 1, epi, Ab, K, Bb, K, M, N, K, 1, bias)
    A, B = Af.astype(np.float64), Bf.astype(np.float64).T
    ref = A @ B + (bias[None, :] if epi == 3 else bias[:, None])
    mag = np.abs(A) @ np.abs(B)
    assert np.all(np.abs(C - ref) <= 2e-5 * mag + 1e-6 * np.abs(bias).max())


@pytest.mark.parametrize("epi,M,N,K", [(1, 40000, 256, 256), (1, 20001, 128, 128), (1, 16500, 48, 64),
                                       (4, 128, 50000, 256), (4, 48, 20001, 128), (4, 119, 16387, 256)])
def test_weight_stationary_kernel(lll, epi, M, N, K):
    """Forward products with at least 16,384 streamed rows run on the
    weight-stationary persistent kernel: the layer's weights stay in shared
    memory while warp-specialised roles stream row tiles through a ring and
    two tensor-memory accumulators.  Epilogue 1 streams A (activations, 128-row
    tiles) against stationary weights; epilogue 4 streams B (256 activation
    rows per tile) against a stationary output layer.  Ragged last tiles and
    N not a multiple of 4 are included."""
    rng = np.random.default_rng(epi * 1000 + M + N)
    Af, Ab = _bf16(rng, (M, K))
    Bf, Bb = _bf16(rng, (N, K), 0.1)
    bias = rng.normal(size=(N if epi == 1 else M)).astype(np.float32)
    lll.lll_set_gemm_kernel("tc")
    C, H = lll.lll_gemm_bf16(0, 1, epi, Ab, K, Bb, K, M, N, K, 1, bias)
    A, B = Af.astype(np.float64), Bf.astype(np.float64).T
    ref = A @ B + (bias[None, :] if epi == 1 else bias[:, None])
    mag = np.abs(A) @ np.abs(B)
    assert np.all(np.abs(C - ref) <= 2e-5 * mag + 1e-6 * np.abs(bias).max())
    if epi == 1:
        h = _bits_to_f(H)
        assert np.all(np.abs(h - _silu(ref)) <= 4e-3 * np.maximum(np.abs(ref), 1.0))
