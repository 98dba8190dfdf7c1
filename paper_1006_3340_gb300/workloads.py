"""Seeded synthetic inputs for the Levy LIBOR Monte Carlo.

This module only builds model inputs: tenor grids, initial forward curves,
volatility tables, NIG parameters, strike grids, path counts and seeds.  It
holds none of the method's arithmetic (no drift, no sampling, no pricing), so
that the CUDA path and the FP64 oracle can both be fed from it without sharing
any computation.

Conventions (Section 2 of the paper, tenor 0 = T_0 < ... < T_N = T_*):
  * ``N`` accrual dates T_k = k*delta, k = 0..N, the terminal date is T_N.
  * The simulated rates are L_m = L(., T_m) for m = 1..n with n = N - 1; the
    spot rate L_0 is known at t = 0.
  * ``L0`` has length N and holds L(0, T_m) for m = 0..N-1.
  * ``lam`` has shape [n*s, n]; ``lam[k, l-1]`` is lambda(t_k, T_l) at the left
    point t_k = k*h of Euler step k, h = delta/s.
  * ``strikes`` has shape [n, n_strikes]; row m-1 holds the strikes of the
    caplet that fixes at T_m.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    N: int
    delta: float
    s: int
    L0: np.ndarray            # [N]
    lam: np.ndarray           # [n*s, n]
    driver: str               # "nig" or "brownian"
    alpha: float = 0.0
    beta: float = 0.0
    dbar: float = 0.0
    mu: Optional[float] = None  # None: martingale drift -dbar*beta/gamma
    a: float = 1.5            # quadrature half-width |x| <= a
    Q: int = 0
    strikes: np.ndarray = None  # [n, ns]
    paths: int = 0
    seed: int = 42
    inst: int = 0

    @property
    def n(self) -> int:
        return self.N - 1

    @property
    def steps(self) -> int:
        return self.n * self.s

    @property
    def h(self) -> float:
        return self.delta / self.s

    def units_per_path(self) -> int:
        """(live rate, step) pairs per path: rate i is live for steps k < i*s."""
        return self.s * self.n * (self.n + 1) // 2

    def with_paths(self, paths: int) -> "Workload":
        return dataclasses.replace(self, paths=int(paths))


def _lam_table(N: int, delta: float, s: int, f) -> np.ndarray:
    """lam[k, l-1] = f(T_l - t_k) for the left point t_k of each Euler step."""
    n = N - 1
    h = delta / s
    k = np.arange(n * s, dtype=np.float64)[:, None]
    T = (np.arange(1, n + 1, dtype=np.float64) * delta)[None, :]
    return np.ascontiguousarray(f(T - k * h), dtype=np.float64)


def _strike_grid(L0: np.ndarray, offsets_bp) -> np.ndarray:
    """ATM = L(0, T_m) of the fixing rate, shifted by the offsets, clamped >= 0."""
    atm = np.asarray(L0[1:], dtype=np.float64)[:, None]
    off = np.asarray(offsets_bp, dtype=np.float64)[None, :] * 1e-4
    return np.ascontiguousarray(np.maximum(atm + off, 0.0))


def small_plain(paths: int = 20000, driver: str = "nig") -> Workload:
    """N=10 semiannual tenors, flat 4 %, lambda = 0.15, NIG(18, -4, 1.0),
    10 steps per period, 32 nodes on |x| <= 1.5, ATM caplets at 9 maturities.
    ``driver="brownian"`` gives the sigma = 0.15 log-normal variant."""
    N, delta, s = 10, 0.5, 10
    L0 = np.full(N, 0.04)
    lam = _lam_table(N, delta, s, lambda tau: np.full_like(tau, 0.15))
    strikes = _strike_grid(L0, [0.0])
    if driver == "brownian":
        return Workload("small_plain_brownian", N, delta, s, L0, lam, "brownian",
                        Q=0, strikes=strikes, paths=paths, seed=42)
    return Workload("small_plain", N, delta, s, L0, lam, "nig", alpha=18.0,
                    beta=-4.0, dbar=1.0, a=1.5, Q=32, strikes=strikes,
                    paths=paths, seed=42)


def large_single(paths: int = 1 << 20) -> Workload:
    """N=40 quarterly tenors (10y), humped curve 0.03 + 0.01(1 - e^{-T/3}),
    lambda = 0.1 + 0.08 e^{-(T_i - t)}, NIG(12, -3, 0.8), 8 steps per period,
    64 nodes on |x| <= 1.5, strikes ATM +- {0, 100, 200} bp."""
    N, delta, s = 40, 0.25, 8
    T = np.arange(N) * delta
    L0 = 0.03 + 0.01 * (1.0 - np.exp(-T / 3.0))
    lam = _lam_table(N, delta, s, lambda tau: 0.1 + 0.08 * np.exp(-tau))
    strikes = _strike_grid(L0, [-200, -100, 0, 100, 200])
    return Workload("large_single", N, delta, s, L0, lam, "nig", alpha=12.0,
                    beta=-3.0, dbar=0.8, a=1.5, Q=64, strikes=strikes,
                    paths=paths, seed=42)


def long_dated(paths: int = 1 << 22) -> Workload:
    """N=120 quarterly tenors (30y), lambda = 0.12 + 0.1 e^{-0.5(T_i - t)},
    NIG(10, -2.5, 1.2), 4 steps per period, 96 nodes, 9 strikes."""
    N, delta, s = 120, 0.25, 4
    T = np.arange(N) * delta
    L0 = 0.03 + 0.01 * (1.0 - np.exp(-T / 3.0))
    lam = _lam_table(N, delta, s, lambda tau: 0.12 + 0.1 * np.exp(-0.5 * tau))
    strikes = _strike_grid(L0, [-200, -150, -100, -50, 0, 50, 100, 150, 200])
    return Workload("long_dated", N, delta, s, L0, lam, "nig", alpha=10.0,
                    beta=-2.5, dbar=1.2, a=1.5, Q=96, strikes=strikes,
                    paths=paths, seed=42)


def batched_instances(n_inst: int = 256, total_paths: int = 1 << 24,
                      seed: int = 42) -> List[Workload]:
    """Uneven independent term structures: N ~ U{8..80}, delta in {0.25, 0.5},
    flat L0 ~ U[0.01, 0.06], lambda = level * e^{-rate (T_i - t)} with level
    ~ U[0.05, 0.25] and rate ~ U[0, 1.5], NIG alpha ~ U[8, 25],
    beta/alpha ~ U[-0.4, 0], dbar = 1, 8 steps per period, 64 nodes, 11
    strikes, path budgets 2^e with e uniform on {12..18} rescaled so that the
    total is exactly ``total_paths``."""
    rng = np.random.default_rng(seed)
    out = []
    exps = rng.integers(12, 19, size=n_inst)
    budget = (2.0 ** exps)
    budget = np.floor(budget * (total_paths / budget.sum())).astype(np.int64)
    budget[-1] += total_paths - budget.sum()
    for q in range(n_inst):
        N = int(rng.integers(8, 81))
        delta = float(rng.choice([0.25, 0.5]))
        lvl0 = float(rng.uniform(0.01, 0.06))
        level = float(rng.uniform(0.05, 0.25))
        rate = float(rng.uniform(0.0, 1.5))
        alpha = float(rng.uniform(8.0, 25.0))
        beta = float(rng.uniform(-0.4, 0.0)) * alpha
        s = 8
        L0 = np.full(N, lvl0)
        lam = _lam_table(N, delta, s, lambda tau, lv=level, r=rate: lv * np.exp(-r * tau))
        span = alpha - abs(beta)
        a = 1.5 if span * 1.5 >= 25.0 else 25.0 / span
        strikes = _strike_grid(L0, [-100, -80, -60, -40, -20, 0, 20, 40, 60, 80, 100])
        out.append(Workload(f"batched_{q}", N, delta, s, L0, lam, "nig", alpha=alpha,
                            beta=beta, dbar=1.0, a=a, Q=64, strikes=strikes,
                            paths=int(budget[q]), seed=seed, inst=q))
    return out


# Zero-coupon bond prices B(0, T) of Table 4.1 (Euro curve, Feb 19 2002),
# T = 0.5, 1.0, ..., 5.0, and the volatility ladder of Section 4.
PAPER_TABLE_4_1_B = np.array([0.9833630, 0.9647388, 0.9435826, 0.9228903, 0.9006922,
                              0.8790279, 0.8568412, 0.8352144, 0.8133497, 0.7920573])
PAPER_LAMBDA_LADDER = np.array([0.20, 0.19, 0.18, 0.17, 0.16, 0.15, 0.14, 0.13, 0.12])


def paper_example(paths: int = 10000, a: float = 30.0, Q: int = 96,
                  offsets_bp=(-200, -100, 0, 100, 200)) -> Workload:
    """Section 4: T_k = k/2 up to T_10 = 5, Table 4.1 discount curve (L(0, T_i)
    from Eq. (i-val) with B(0, T_0) = 1), lambda ladder 0.20 ... 0.12,
    NIG alpha = dbar = 1.5, beta = mu = 0, 5 steps per period.  The paper's
    strike grid is not printed; ``offsets_bp`` chooses one."""
    N, delta, s = 10, 0.5, 5
    B = np.concatenate([[1.0], PAPER_TABLE_4_1_B])
    L0 = (B[:-1] / B[1:] - 1.0) / delta
    lam = np.ascontiguousarray(np.tile(PAPER_LAMBDA_LADDER[None, :], ((N - 1) * s, 1)))
    strikes = _strike_grid(L0, list(offsets_bp))
    return Workload("paper_example", N, delta, s, L0, lam, "nig", alpha=1.5, beta=0.0,
                    dbar=1.5, mu=0.0, a=a, Q=Q, strikes=strikes, paths=paths, seed=42)


def tiny(N: int = 4, s: int = 3, Q: int = 8, paths: int = 64, driver: str = "nig",
         seed: int = 7) -> Workload:
    """A few rates and steps for exhaustive checks."""
    delta = 0.5
    L0 = 0.03 + 0.005 * np.arange(N)
    lam = _lam_table(N, delta, s, lambda tau: 0.12 + 0.05 * np.exp(-tau))
    strikes = _strike_grid(L0, [-50, 0, 50])
    if driver == "brownian":
        return Workload("tiny_brownian", N, delta, s, L0, lam, "brownian", Q=0,
                        strikes=strikes, paths=paths, seed=seed)
    return Workload("tiny", N, delta, s, L0, lam, "nig", alpha=9.0, beta=-2.0, dbar=1.0,
                    a=1.5, Q=Q, strikes=strikes, paths=paths, seed=seed)


def by_name(name: str, **kw) -> Workload:
    return {"small_plain": small_plain, "large_single": large_single,
            "long_dated": long_dated, "paper_example": paper_example,
            "tiny": tiny}[name](**kw)
