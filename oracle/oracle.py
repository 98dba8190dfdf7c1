"""ctypes wrapper of the FP64 C oracle (lll_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the package smoke check and the
CPU-baseline leg of the benchmark are its only users.  It shares no code with
the CUDA library.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "lll_oracle.c")
_LIB = os.path.join(_BUILD, "liblll_oracle.so")

FULL, PICARD, FROZEN = 0, 1, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: no -march, no intrinsics)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class _Model(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("s", ctypes.c_int32), ("Q", ctypes.c_int32),
                ("driver", ctypes.c_int32), ("delta", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("dbar", ctypes.c_double), ("mu", ctypes.c_double),
                ("L0", ctypes.c_void_p), ("lam", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("W", ctypes.c_void_p)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_simulate.restype = ctypes.c_int
        _lib.oracle_simulate_list.restype = ctypes.c_int
        _lib.oracle_increments.restype = ctypes.c_int
        _lib.oracle_drift.restype = ctypes.c_int
        _lib.oracle_frozen_drift.restype = ctypes.c_int
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleModel:
    """Holds FP64 copies of the inputs alive for the duration of the calls."""

    def __init__(self, wl, nodes=None, weights=None):
        self.wl = wl
        self.L0 = np.ascontiguousarray(wl.L0, dtype=np.float64)
        self.lam = np.ascontiguousarray(wl.lam, dtype=np.float64)
        if wl.driver == "brownian":
            self.x = np.zeros(1)
            self.W = np.zeros(1)
            Q = 0
        else:
            self.x = np.ascontiguousarray(nodes, dtype=np.float64)
            self.W = np.ascontiguousarray(weights, dtype=np.float64)
            Q = len(self.x)
        mu = float("nan") if wl.mu is None else float(wl.mu)
        self.c = _Model(wl.N, wl.s, Q, 1 if wl.driver == "brownian" else 0, wl.delta,
                        wl.alpha, wl.beta, wl.dbar, mu, _ptr(self.L0), _ptr(self.lam),
                        _ptr(self.x), _ptr(self.W))

    @property
    def n(self):
        return self.wl.N - 1


def simulate(model: OracleModel, scheme: int, path0: int = 0, npaths: Optional[int] = None,
             strikes=None, want_snap: bool = False, threads: Optional[int] = None,
             seed: Optional[int] = None, inst: Optional[int] = None):
    """Run one scheme.  Returns dict with payoff sums, prices, standard errors,
    optional log-rate snapshots snap[p, m-1, l-1] = log L_l(T_m) (l >= m) and
    the per-path minimum |IG acceptance margin|."""
    lib = _load()
    wl = model.wl
    n = model.n
    npaths = wl.paths if npaths is None else int(npaths)
    strikes = np.ascontiguousarray(wl.strikes if strikes is None else strikes, dtype=np.float64)
    ns = strikes.shape[1]
    s1 = np.zeros((n, ns))
    s2 = np.zeros((n, ns))
    snap = np.full((npaths, n, n), np.nan) if want_snap else None
    mm = np.zeros(npaths)
    threads = threads or os.cpu_count() or 1
    seed = wl.seed if seed is None else seed
    inst = wl.inst if inst is None else inst
    st = lib.oracle_simulate(ctypes.byref(model.c), ctypes.c_int(scheme),
                             ctypes.c_uint64(seed), ctypes.c_uint32(inst),
                             ctypes.c_uint64(path0), ctypes.c_uint64(npaths), ctypes.c_int(ns),
                             _ptr(strikes), _ptr(s1), _ptr(s2), _ptr(snap), _ptr(mm),
                             ctypes.c_int(threads))
    if st != 0:
        raise RuntimeError(f"oracle_simulate failed: {st}")
    return dict(sum=s1, sumsq=s2, snap=snap, min_margin=mm, npaths=npaths,
                **moments(s1, s2, npaths))


def simulate_paths(model: OracleModel, scheme: int, paths, strikes=None, threads=None,
                   seed=None, inst=None):
    """Like :func:`simulate` for an explicit list of path indices; returns the
    snapshots snap[q, m-1, l-1] of path paths[q] and the payoff sums."""
    lib = _load()
    wl = model.wl
    n = model.n
    plist = np.ascontiguousarray(paths, dtype=np.uint64)
    npaths = len(plist)
    strikes = np.ascontiguousarray(wl.strikes if strikes is None else strikes, dtype=np.float64)
    ns = strikes.shape[1]
    s1 = np.zeros((n, ns))
    s2 = np.zeros((n, ns))
    snap = np.full((npaths, n, n), np.nan)
    mm = np.zeros(npaths)
    threads = threads or os.cpu_count() or 1
    seed = wl.seed if seed is None else seed
    inst = wl.inst if inst is None else inst
    st = lib.oracle_simulate_list(ctypes.byref(model.c), ctypes.c_int(scheme), ctypes.c_uint64(seed),
                                  ctypes.c_uint32(inst), plist.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_uint64(npaths), ctypes.c_int(ns), _ptr(strikes), _ptr(s1),
                                  _ptr(s2), _ptr(snap), _ptr(mm), ctypes.c_int(threads))
    if st != 0:
        raise RuntimeError(f"oracle_simulate_list failed: {st}")
    return dict(sum=s1, sumsq=s2, snap=snap, min_margin=mm, npaths=npaths)


def moments(s1, s2, npaths):
    """Price = sample mean of the payoff; standard error from the
    (P-1)-normalised sample variance."""
    mean = s1 / npaths
    var = np.maximum(s2 / npaths - mean * mean, 0.0) * npaths / max(npaths - 1, 1)
    return dict(price=mean, se=np.sqrt(var / npaths))


def increments(model: OracleModel, path0: int, npaths: int, seed=None, inst=None):
    lib = _load()
    wl = model.wl
    S = wl.steps
    dH = np.zeros((npaths, S))
    mg = np.zeros((npaths, S))
    seed = wl.seed if seed is None else seed
    inst = wl.inst if inst is None else inst
    st = lib.oracle_increments(ctypes.byref(model.c), ctypes.c_uint64(seed), ctypes.c_uint32(inst),
                               ctypes.c_uint64(path0), ctypes.c_uint64(npaths), _ptr(dH), _ptr(mg))
    if st != 0:
        raise RuntimeError("oracle_increments failed")
    return dH, mg


def drift(model: OracleModel, k: int, i: int, w) -> float:
    lib = _load()
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = ctypes.c_double()
    st = lib.oracle_drift(ctypes.byref(model.c), ctypes.c_int(k), ctypes.c_int(i), _ptr(w),
                          ctypes.byref(out))
    if st != 0:
        raise RuntimeError("oracle_drift failed")
    return out.value


def frozen_drift(model: OracleModel):
    lib = _load()
    S, n = model.wl.steps, model.n
    b0 = np.zeros((S, n))
    D0 = np.zeros((S + 1, n))
    st = lib.oracle_frozen_drift(ctypes.byref(model.c), _ptr(b0), _ptr(D0))
    if st != 0:
        raise RuntimeError("oracle_frozen_drift failed")
    return b0, D0


def philox(ctr, key):
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.oracle_philox(c, k, o)
    return [o[0], o[1], o[2], o[3]]


def discount_terminal(wl) -> float:
    """B(0, T_N) = prod_{m<N} (1 + delta L(0, T_m))^{-1} (Eq. (i-val) inverted)."""
    return float(np.prod(1.0 / (1.0 + wl.delta * np.asarray(wl.L0))))


def discount(wl, k: int) -> float:
    return float(np.prod(1.0 / (1.0 + wl.delta * np.asarray(wl.L0[:k]))))


def swaption_prices(wl, snap, strikes=None):
    """Co-terminal payer swaptions priced on simulated paths (Section 1 names
    swaptions as the multi-LIBOR products without closed forms).

    The swaption expiring at T_m exercises into the swap over [T_m, T_N]:
    fixed rate K against L, both legs paying at T_{m+1} .. T_N.  Its value at
    T_m, written with the bond prices of that date,
        B(T_m, T_j) = prod_{l=m}^{j-1} 1 / (1 + delta L_l(T_m)),
    is V_m = (1 - B(T_m, T_N) - K delta sum_{j=m+1}^{N} B(T_m, T_j))^+.  Under
    the terminal measure its price is B(0, T_N) E[V_m / B(T_m, T_N)].

    snap[p, m-1, l-1] = log L_l(T_m) (l >= m) of the paths; strikes [n][ns].
    Returns prices [n][ns]."""
    n, d = wl.N - 1, wl.delta
    strikes = np.asarray(wl.strikes if strikes is None else strikes, dtype=np.float64)
    BN = discount_terminal(wl)
    out = np.zeros((n, strikes.shape[1]))
    for m in range(1, n + 1):
        L = np.exp(np.asarray(snap[:, m - 1, m - 1:], dtype=np.float64))  # L_m .. L_n at T_m
        # B(T_m, T_j) for j = m+1 .. N: running product of the discount factors
        bonds = np.cumprod(1.0 / (1.0 + d * L), axis=1)
        for q in range(strikes.shape[1]):
            V = np.maximum(1.0 - bonds[:, -1] - strikes[m - 1, q] * d * bonds.sum(axis=1), 0.0)
            out[m - 1, q] = BN * np.mean(V / bonds[:, -1])
    return out
