"""ctypes binding of liblll.so (include/lll.h).  Argument marshalling only:
every step of the simulation runs in the library's CUDA kernels.

The library must have been built (``paper_1006_3340_gb300.build.build()`` or
``__graft_entry__.build()``); loading fails loudly otherwise.  There is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

import numpy as np

from . import build as _build

LLL_OK, LLL_EINVAL, LLL_EDOMAIN, LLL_ECUDA, LLL_ETIMEOUT, LLL_ENOMEM, LLL_ESTATE, LLL_EUNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7
LLL_FULL, LLL_PICARD, LLL_MLP, LLL_FROZEN, LLL_EXPAND1, LLL_EXPAND2 = 0, 1, 2, 3, 4, 5
LLL_DRIVER_NIG, LLL_DRIVER_BROWNIAN = 0, 1
SCHEMES = {"full": LLL_FULL, "picard": LLL_PICARD, "mlp": LLL_MLP, "frozen": LLL_FROZEN,
           "expand1": LLL_EXPAND1, "expand2": LLL_EXPAND2}


class LLLError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"liblll status {code}: {msg}")
        self.code = code


class lll_mlp_cfg(ctypes.Structure):
    _fields_ = [("hidden", ctypes.c_int), ("layers", ctypes.c_int), ("train_paths", ctypes.c_uint64),
                ("records_per_path", ctypes.c_int), ("epochs", ctypes.c_int), ("batch", ctypes.c_int),
                ("lr", ctypes.c_double), ("lr_final", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("head", ctypes.c_int)]


class lll_nig(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("delta", ctypes.c_double), ("mu", ctypes.c_double)]


class lll_instance(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("tenor_delta", ctypes.c_double), ("L0", ctypes.c_void_p),
                ("steps_per_period", ctypes.c_int), ("lambda_", ctypes.c_void_p), ("driver", ctypes.c_int),
                ("nig", lll_nig), ("Q", ctypes.c_int), ("nodes", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("n_strikes", ctypes.c_int), ("strikes", ctypes.c_void_p), ("paths", ctypes.c_uint64)]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)


def library_path() -> str:
    return _build.LIB


def load():
    """Load liblll.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"liblll.so not built ({path}); run paper_1006_3340_gb300.build.build()")
    lib = ctypes.CDLL(path)
    V, I, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64
    sigs = {
        "lll_init": (I, [ctypes.POINTER(V), I, ctypes.c_double, _dp, I, _dp, I, lll_nig, I, _dp, _dp, V]),
        "lll_set_strikes": (I, [V, I, _dp]),
        "lll_set_product": (I, [V, I]),
        "lll_set_snapshots": (I, [V, U64, U64]),
        "lll_simulate": (I, [V, I, U64, U64, U64]),
        "lll_simulate_noalloc": (I, [V, I, U64, U64, U64, V]),
        "lll_get_sums": (I, [V, _dp, _dp, ctypes.POINTER(U64)]),
        "lll_price_caplets": (I, [V, _dp, _dp]),
        "lll_get_paths": (I, [V, U64, U64, _fp]),
        "lll_set_launch": (I, [V, I, I, I, I, I]),
        "lll_set_mapping": (I, [V, I, I]),
        "lll_kernel_ms": (I, [V, _fp, _fp]),
        "lll_build_nig_quadrature": (I, [lll_nig, ctypes.c_double, I, _dp, _dp]),
        "lll_mlp_init": (I, [V, I, I, U64]),
        "lll_mlp_init_head": (I, [V, I, I, I, U64]),
        "lll_mlp_shape": (I, [V, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "lll_mlp_train": (I, [V, ctypes.POINTER(lll_mlp_cfg), _dp]),
        "lll_mlp_layout": (I, [V, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(I), ctypes.POINTER(I),
                               ctypes.POINTER(ctypes.c_size_t)]),
        "lll_mlp_params": (I, [V, I, _fp, ctypes.c_size_t, _fp]),
        "lll_mlp_eval": (I, [V, _fp, _fp, I, _fp, _fp, _dp]),
        "lll_mlp_save": (I, [V, ctypes.c_char_p]),
        "lll_mlp_load": (I, [V, ctypes.c_char_p]),
        "lll_mlp_set_kernel": (I, [V, I]),
        "lll_inject": (I, [V, I]),
        "lll_philox_words": (I, [V, U64, U64, V]),
        "lll_set_gemm_kernel": (I, [I]),
        "lll_gemm_bf16": (I, [I, I, I, V, I, V, I, I, I, I, I, V, V, V, V]),
        "lll_measure_pipe_rates": (I, [_dp, I]),
        "lll_batch_init": (I, [ctypes.POINTER(V), I, ctypes.POINTER(lll_instance), V]),
        "lll_batch_set_launch": (I, [V, I, I, I, I, I]),
        "lll_batch_use_graph": (I, [V, I]),
        "lll_batch_simulate": (I, [V, I, U64]),
        "lll_batch_prices": (I, [V, I, _dp, _dp]),
        "lll_batch_kernel_ms": (I, [V, _fp]),
        "lll_batch_set_snapshots": (I, [V, I, U64, U64]),
        "lll_batch_get_paths": (I, [V, I, U64, U64, _fp]),
        "lll_batch_destroy": (None, [V]),
        "lll_last_error": (ctypes.c_char_p, [V]),
        "lll_destroy": (None, [V]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, ctx=None, allow=(LLL_OK,)):
    if rc not in allow:
        msg = load().lll_last_error(ctx)
        raise LLLError(rc, msg.decode() if msg else "")
    return rc


# ---- the C entry points, same names ----------------------------------------
def lll_build_nig_quadrature(alpha, beta, delta, xmax, Q, mu=float("nan")):
    lib = load()
    x = np.zeros(Q)
    w = np.zeros(Q)
    _check(lib.lll_build_nig_quadrature(lll_nig(alpha, beta, delta, mu), float(xmax), int(Q), _d(x), _d(w)))
    return x, w


def lll_init(N, delta, L0, s, lam, driver, nig=(0.0, 0.0, 0.0, float("nan")), nodes=None,
             weights=None, stream: int = 0, allow_domain_warning: bool = True):
    """Returns (ctx handle, status).  ``stream`` is a cudaStream_t as int."""
    lib = load()
    L0 = _f64(L0)
    lam = _f64(lam)
    if nodes is None:
        nodes, weights, Q = np.zeros(1), np.zeros(1), 0
    else:
        nodes, weights = _f64(nodes), _f64(weights)
        Q = len(nodes)
    ctx = ctypes.c_void_p()
    mu = float("nan") if nig[3] is None else float(nig[3])
    rc = lib.lll_init(ctypes.byref(ctx), int(N), float(delta), _d(L0), int(s), _d(lam), int(driver),
                      lll_nig(float(nig[0]), float(nig[1]), float(nig[2]), mu), int(Q), _d(nodes),
                      _d(weights), ctypes.c_void_p(stream or None))
    allowed = (LLL_OK, LLL_EDOMAIN) if allow_domain_warning else (LLL_OK,)
    _check(rc, None, allowed)
    return ctx, rc


def lll_set_strikes(ctx, strikes):
    strikes = _f64(strikes)
    _check(load().lll_set_strikes(ctx, int(strikes.shape[1]), _d(strikes)), ctx)


def lll_set_snapshots(ctx, count, stride=1):
    _check(load().lll_set_snapshots(ctx, int(count), int(stride)), ctx)


def lll_simulate(ctx, scheme, first_path, paths, seed):
    _check(load().lll_simulate(ctx, int(scheme), int(first_path), int(paths), int(seed)), ctx)


def lll_simulate_noalloc(ctx, scheme, first_path, paths, seed, d_sums: int):
    """``d_sums``: device address of n * n_strikes * 2 doubles owned by the caller."""
    _check(load().lll_simulate_noalloc(ctx, int(scheme), int(first_path), int(paths), int(seed),
                                       ctypes.c_void_p(d_sums)), ctx)


def lll_get_sums(ctx, n, ns):
    s1 = np.zeros((n, ns))
    s2 = np.zeros((n, ns))
    cnt = ctypes.c_uint64()
    _check(load().lll_get_sums(ctx, _d(s1), _d(s2), ctypes.byref(cnt)), ctx)
    return s1, s2, cnt.value


def lll_price_caplets(ctx, n, ns):
    p = np.zeros((n, ns))
    se = np.zeros((n, ns))
    _check(load().lll_price_caplets(ctx, _d(p), _d(se)), ctx)
    return p, se


def lll_get_paths(ctx, n, first, count):
    out = np.zeros((count, n, n), dtype=np.float32)
    _check(load().lll_get_paths(ctx, int(first), int(count), out.ctypes.data_as(_fp)), ctx)
    return out


def lll_set_launch(ctx, threads=0, blocks_per_sm=0, chunk_rows=0, paths_per_thread=0, lanes_per_path=0):
    _check(load().lll_set_launch(ctx, int(threads), int(blocks_per_sm), int(chunk_rows),
                                 int(paths_per_thread), int(lanes_per_path)), ctx)


LLL_MAP_PATH, LLL_MAP_TENOR, LLL_MAP_STEP = 0, 1, 2


def lll_set_mapping(ctx, mapping, lanes=0):
    """mapping: "path" (one lane per path), "tenor" (``lanes`` lanes per path) or
    "step" (Picard: the Euler steps of a path in parallel)."""
    m = {"path": LLL_MAP_PATH, "tenor": LLL_MAP_TENOR, "step": LLL_MAP_STEP}.get(mapping, mapping)
    _check(load().lll_set_mapping(ctx, int(m), int(lanes)), ctx)


def lll_kernel_ms(ctx):
    a = ctypes.c_float()
    b = ctypes.c_float()
    _check(load().lll_kernel_ms(ctx, ctypes.byref(a), ctypes.byref(b)), ctx)
    return a.value, b.value


def lll_mlp_init(ctx, hidden, layers, seed=0, head=0):
    _check(load().lll_mlp_init_head(ctx, int(hidden), int(layers), int(head), int(seed)), ctx)


def lll_mlp_init_head(ctx, hidden, layers, head, seed=0):
    _check(load().lll_mlp_init_head(ctx, int(hidden), int(layers), int(head), int(seed)), ctx)


def lll_mlp_shape(ctx):
    """(head, outputs) of the context's network."""
    h, o = ctypes.c_int(), ctypes.c_int()
    _check(load().lll_mlp_shape(ctx, ctypes.byref(h), ctypes.byref(o)), ctx)
    return h.value, o.value


def lll_mlp_train(ctx, hidden=128, layers=3, train_paths=1 << 16, records_per_path=8, epochs=4,
                  batch=8192, lr=2e-3, lr_final=2e-4, seed=7, head=0):
    cfg = lll_mlp_cfg(int(hidden), int(layers), int(train_paths), int(records_per_path), int(epochs),
                      int(batch), float(lr), float(lr_final), int(seed), int(head))
    loss = ctypes.c_double()
    _check(load().lll_mlp_train(ctx, ctypes.byref(cfg), ctypes.byref(loss)), ctx)
    return loss.value


def lll_mlp_layout(ctx, layers):
    n = ctypes.c_size_t()
    ind = ctypes.c_int()
    inp = ctypes.c_int()
    offs = (ctypes.c_size_t * (2 * layers + 2))()
    _check(load().lll_mlp_layout(ctx, ctypes.byref(n), ctypes.byref(ind), ctypes.byref(inp), offs), ctx)
    return n.value, ind.value, inp.value, list(offs)


def lll_mlp_params(ctx, direction, params=None, count=None, scales=None):
    """direction 0: returns (params, scales); 1: sets them."""
    if direction == 0:
        p = np.zeros(count, dtype=np.float32)
        sc = np.zeros(5, dtype=np.float32)
        _check(load().lll_mlp_params(ctx, 0, p.ctypes.data_as(_fp), p.size, sc.ctypes.data_as(_fp)), ctx)
        return p, sc
    p = np.ascontiguousarray(params, dtype=np.float32)
    sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float32)
    _check(load().lll_mlp_params(ctx, 1, p.ctypes.data_as(_fp), p.size,
                                 None if sc is None else sc.ctypes.data_as(_fp)), ctx)


def lll_mlp_eval(ctx, x, y=None, n_params=None, want_grads=False):
    x = np.ascontiguousarray(x, dtype=np.float32)
    rows = x.shape[0]
    head, outputs = lll_mlp_shape(ctx)
    out = np.zeros((rows, outputs) if head else rows, dtype=np.float32)
    yy = None if y is None else np.ascontiguousarray(y, dtype=np.float32)
    g = np.zeros(n_params, dtype=np.float32) if want_grads else None
    loss = ctypes.c_double()
    _check(load().lll_mlp_eval(ctx, x.ctypes.data_as(_fp), None if yy is None else yy.ctypes.data_as(_fp),
                               rows, out.ctypes.data_as(_fp), None if g is None else g.ctypes.data_as(_fp),
                               ctypes.byref(loss)), ctx)
    return out, g, loss.value


def lll_mlp_save(ctx, path):
    _check(load().lll_mlp_save(ctx, str(path).encode()), ctx)


def lll_mlp_load(ctx, path):
    _check(load().lll_mlp_load(ctx, str(path).encode()), ctx)


MLP_KERNELS = {"auto": 0, "warp": 1, "tc": 2, "layered": 3}
LLL_INJECT_NONE, LLL_INJECT_MMA_STALL = 0, 1
PRODUCTS = {"caplet": 0, "swaption": 1}


def lll_set_product(ctx, product):
    """Payoff at each T_m: "caplet" (default) or "swaption" (co-terminal payer)."""
    _check(load().lll_set_product(ctx, PRODUCTS[product] if isinstance(product, str) else int(product)), ctx)


def lll_inject(ctx, what):
    """Failure-detection testing (see include/lll.h)."""
    _check(load().lll_inject(ctx, int(what)), ctx)


def lll_mlp_set_kernel(ctx, kind):
    """Kernel of LLL_MLP: "auto", "warp" (mma.sync), "tc" (tcgen05 + TMEM) or "layered"."""
    _check(load().lll_mlp_set_kernel(ctx, MLP_KERNELS[kind] if isinstance(kind, str) else int(kind)), ctx)


def lll_batch_init(instances, stream: int = 0):
    """instances: list of (workload, nodes, weights).  Returns (handle, keepalive)."""
    lib = load()
    keep = []
    arr = (lll_instance * len(instances))()
    for q, (wl, x, W) in enumerate(instances):
        L0, lam, st = _f64(wl.L0), _f64(wl.lam), _f64(wl.strikes)
        x, W = _f64(x), _f64(W)
        keep += [L0, lam, st, x, W]
        mu = float("nan") if wl.mu is None else float(wl.mu)
        arr[q] = lll_instance(wl.N, wl.delta, L0.ctypes.data, wl.s, lam.ctypes.data, LLL_DRIVER_NIG,
                              lll_nig(wl.alpha, wl.beta, wl.dbar, mu), len(x), x.ctypes.data, W.ctypes.data,
                              st.shape[1], st.ctypes.data, int(wl.paths))
    h = ctypes.c_void_p()
    _check(lib.lll_batch_init(ctypes.byref(h), len(instances), arr, ctypes.c_void_p(stream or None)))
    return h, keep


def lll_batch_set_launch(b, threads=0, blocks_per_sm=0, chunk_rows=0, paths_per_thread=0, scheme=-1):
    """Launch shape of ``scheme`` (LLL_FULL, LLL_PICARD, a name, or -1: both)."""
    sc = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    _check(load().lll_batch_set_launch(b, sc, int(threads), int(blocks_per_sm), int(chunk_rows),
                                       int(paths_per_thread)))


def lll_batch_use_graph(b, enable=True):
    _check(load().lll_batch_use_graph(b, 1 if enable else 0))


def lll_batch_simulate(b, scheme, seed):
    _check(load().lll_batch_simulate(b, int(scheme), int(seed)))


def lll_batch_prices(b, q, n, ns):
    p = np.zeros((n, ns))
    se = np.zeros((n, ns))
    _check(load().lll_batch_prices(b, int(q), _d(p), _d(se)))
    return p, se


def lll_batch_set_snapshots(b, q, count, stride=1):
    _check(load().lll_batch_set_snapshots(b, int(q), int(count), int(stride)))


def lll_batch_get_paths(b, q, n, first, count):
    """log L_l(T_m) of recorded snapshots [first, first+count) of instance q: [count, n, n]."""
    out = np.zeros((count, n, n), dtype=np.float32)
    _check(load().lll_batch_get_paths(b, int(q), int(first), int(count), out.ctypes.data_as(_fp)))
    return out


def lll_batch_kernel_ms(b):
    ms = ctypes.c_float()
    _check(load().lll_batch_kernel_ms(b, ctypes.byref(ms)))
    return ms.value


def lll_batch_destroy(b):
    if b:
        load().lll_batch_destroy(b)


def lll_philox_words(counters, seed):
    """Device Philox-4x32-10 output words [count][4] (uint32) for counters [count][4]."""
    ctr = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(ctr)
    _check(load().lll_philox_words(ctr.ctypes.data, ctr.shape[0], int(seed) & (2 ** 64 - 1), out.ctypes.data))
    return out


def lll_set_gemm_kernel(kind):
    """Process-wide GEMM kernel of the learned compensator: "tc" (tcgen05, default) or "mma_sync"."""
    k = {"tc": 0, "mma_sync": 1}.get(kind, kind)
    _check(load().lll_set_gemm_kernel(int(k)))


def lll_gemm_bf16(ta, tb, epi, A_bits, lda, B_bits, ldb, M, N, K, splits=1, bias=None, Zin=None):
    """One product of the current GEMM kernel on host arrays (uint16 BF16 bits).
    Returns C [M, N] (FP32) and, for epi 1/2, H [M, N] (uint16 BF16 bits)."""
    A = np.ascontiguousarray(A_bits, dtype=np.uint16)
    B = np.ascontiguousarray(B_bits, dtype=np.uint16)
    C = np.zeros((M, N), dtype=np.float32)
    H = np.zeros((M, N), dtype=np.uint16) if epi in (1, 2) else None
    b = np.ascontiguousarray(bias, dtype=np.float32) if bias is not None else None
    z = np.ascontiguousarray(Zin, dtype=np.float32) if Zin is not None else None
    ptr = lambda a: a.ctypes.data if a is not None else None  # noqa: E731
    _check(load().lll_gemm_bf16(int(ta), int(tb), int(epi), ptr(A), int(lda), ptr(B), int(ldb), int(M), int(N),
                                int(K), int(splits), ptr(b), ptr(z), ptr(C), ptr(H)))
    return C, H


PIPE_RATE_NAMES = ("tanh", "ex2", "rcp", "ffma2_lane_ops", "ffma_lane_ops")


def lll_measure_pipe_rates(count=5):
    """Measured results per SM per clock: {name: rate} (see include/lll.h)."""
    r = np.zeros(count)
    _check(load().lll_measure_pipe_rates(_d(r), int(count)))
    return {k: float(v) for k, v in zip(PIPE_RATE_NAMES, r)}


def lll_last_error(ctx=None) -> str:
    msg = load().lll_last_error(ctx)
    return msg.decode() if msg else ""


def lll_destroy(ctx):
    if ctx:
        load().lll_destroy(ctx)


# ---- convenience wrapper ---------------------------------------------------
class LevyLibor:
    """One model context (a workload from :mod:`workloads`) on the current CUDA
    device and a caller-chosen stream."""

    def __init__(self, wl, nodes=None, weights=None, stream: int = 0):
        self.wl = wl
        self.n = wl.n
        if wl.driver == "nig":
            if nodes is None:
                nodes, weights = lll_build_nig_quadrature(wl.alpha, wl.beta, wl.dbar, wl.a, wl.Q)
            drv = LLL_DRIVER_NIG
            nig = (wl.alpha, wl.beta, wl.dbar, float("nan") if wl.mu is None else wl.mu)
        else:
            drv, nig, nodes, weights = LLL_DRIVER_BROWNIAN, (0.0, 0.0, 0.0, float("nan")), None, None
        self.ctx, self.init_status = lll_init(wl.N, wl.delta, wl.L0, wl.s, wl.lam, drv, nig, nodes,
                                              weights, stream)
        self.ns = wl.strikes.shape[1]
        lll_set_strikes(self.ctx, wl.strikes)

    def set_strikes(self, strikes):
        lll_set_strikes(self.ctx, strikes)
        self.ns = np.asarray(strikes).shape[1]

    def set_product(self, product):
        lll_set_product(self.ctx, product)

    def simulate(self, scheme="picard", paths=None, first_path=0, seed=None, snapshots=0,
                 snapshot_stride=1):
        sch = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        lll_set_snapshots(self.ctx, snapshots, snapshot_stride)
        lll_simulate(self.ctx, sch, first_path, self.wl.paths if paths is None else paths,
                     self.wl.seed if seed is None else seed)

    def prices(self):
        return lll_price_caplets(self.ctx, self.n, self.ns)

    def sums(self):
        return lll_get_sums(self.ctx, self.n, self.ns)

    def paths(self, first, count):
        return lll_get_paths(self.ctx, self.n, first, count)

    def kernel_ms(self):
        return lll_kernel_ms(self.ctx)

    def set_launch(self, threads=0, blocks_per_sm=0, chunk_rows=0, paths_per_thread=0, lanes_per_path=0):
        lll_set_launch(self.ctx, threads, blocks_per_sm, chunk_rows, paths_per_thread, lanes_per_path)

    def set_mapping(self, mapping, lanes=0):
        lll_set_mapping(self.ctx, mapping, lanes)

    def close(self):
        if self.ctx:
            lll_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
