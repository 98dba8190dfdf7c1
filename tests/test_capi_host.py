"""Host-side checks of liblll.so that need no GPU: the library builds and
loads, exports every function include/lll.h declares, rejects invalid input
before touching the device, and its FP64 Gauss-rule builder (a host
computation) agrees with the oracle's independently written one."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import quadrature
from paper_1006_3340_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lll():
    libbuild.build()
    from paper_1006_3340_gb300 import lll as mod

    mod.load()
    return mod


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b(lll_[a-z0-9_]+)\s*\(",
                                src, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(lll):
    names = _declared_functions()
    assert "lll_init" in names and "lll_simulate" in names and "lll_price_caplets" in names
    lib = ctypes.CDLL(lll.library_path())
    for name in names:
        assert hasattr(lib, name), name


def test_binding_has_same_names(lll):
    for name in _declared_functions():
        assert hasattr(lll, name), name


@pytest.mark.parametrize("alpha,beta,dbar,a,Q", [(18.0, -4.0, 1.0, 1.5, 32), (12.0, -3.0, 0.8, 1.5, 64),
                                                 (10.0, -2.5, 1.2, 1.5, 96), (1.5, 0.0, 1.5, 30.0, 96),
                                                 (9.0, -2.0, 1.0, 1.5, 8)])
def test_quadrature_builder_matches_oracle(lll, alpha, beta, dbar, a, Q):
    x, W = lll.lll_build_nig_quadrature(alpha, beta, dbar, a, Q)
    xo, Wo = quadrature.gauss_rule(alpha, beta, dbar, a, Q)
    assert np.allclose(x, xo, rtol=0, atol=1e-12 * a)
    assert np.all(np.abs(W - Wo) <= 1e-9 * Wo + 1e-13 * Wo.sum())


def _base():
    from paper_1006_3340_gb300 import workloads
    wl = workloads.tiny(N=4, s=2, Q=8)
    x, W = quadrature.rule_for(wl)
    return wl, x, W


@pytest.mark.parametrize("mutate,code", [
    (lambda d: d.update(N=1), -1),
    (lambda d: d.update(delta=0.0), -1),
    (lambda d: d.update(delta=float("nan")), -1),
    (lambda d: d["L0"].__setitem__(2, -0.01), -1),
    (lambda d: d["L0"].__setitem__(0, float("inf")), -1),
    (lambda d: d["lam"].__setitem__((1, 1), float("nan")), -1),
    (lambda d: d.update(s=0), -1),
    (lambda d: d["x"].__setitem__(3, 0.0), -1),
    (lambda d: d.update(nig=(2.0, 3.0, 1.0, float("nan"))), -1),
    (lambda d: d.update(nig=(9.0, -2.0, -1.0, float("nan"))), -1),
    (lambda d: d.update(driver=7), -1),
    (lambda d: d.update(x=np.linspace(-1, 1, 130) + 1e-3, W=np.ones(130)), -7),
])
def test_init_rejects_invalid_input_on_host(lll, mutate, code):
    wl, x, W = _base()
    d = dict(N=wl.N, delta=wl.delta, L0=wl.L0.copy(), s=wl.s, lam=wl.lam.copy(), driver=0,
             nig=(wl.alpha, wl.beta, wl.dbar, float("nan")), x=x.copy(), W=W.copy())
    mutate(d)
    with pytest.raises(lll.LLLError) as e:
        lll.lll_init(d["N"], d["delta"], d["L0"], d["s"], d["lam"], d["driver"], d["nig"], d["x"], d["W"])
    assert e.value.code == code
    assert lll.load().lll_last_error(None)


def test_quadrature_builder_rejects_bad_input(lll):
    for args in [(2.0, 3.0, 1.0, 1.5, 8), (9.0, -2.0, 1.0, -1.0, 8), (9.0, -2.0, 1.0, 1.5, 0)]:
        with pytest.raises(lll.LLLError):
            lll.lll_build_nig_quadrature(*args)
    with pytest.raises(lll.LLLError) as e:
        lll.lll_build_nig_quadrature(9.0, -2.0, 1.0, 1.5, 129)
    assert e.value.code == -7


def test_calls_on_null_context_fail_cleanly(lll):
    lib = lll.load()
    assert lib.lll_simulate(None, 1, 0, 10, 42) == -1
    assert lib.lll_set_strikes(None, 1, None) == -1
    lib.lll_destroy(None)


def test_batch_calls_on_null_handle_fail_cleanly(lll):
    """The batch entry points check their handle and arguments before any CUDA
    call (so these run without a GPU)."""
    lib = lll.load()
    assert lib.lll_batch_init(None, 1, None, None) == -1
    assert lib.lll_batch_set_launch(None, -1, 128, 0, 0, 2) == -1
    assert lib.lll_batch_use_graph(None, 1) == -1
    assert lib.lll_batch_simulate(None, lll.LLL_FULL, 42) == -1
    assert lib.lll_batch_prices(None, 0, None, None) == -1
    assert lib.lll_batch_set_snapshots(None, 0, 1, 1) == -1
    assert lib.lll_batch_get_paths(None, 0, 0, 1, None) == -1
    assert lib.lll_batch_kernel_ms(None, None) == -1
    lib.lll_batch_destroy(None)
