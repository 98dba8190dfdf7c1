"""Closed forms the Monte Carlo is checked against (FP64, oracle side).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the
benchmark).

  * NIG cumulant kappa(u) (Section 4; the general beta, mu form is the
    standard NIG cumulant, the paper prints the beta = mu = 0 case).
  * The product expansion of Eq. (product) turned into the exact drift by
    inclusion-exclusion over subsets, and its truncations: the first-order
    approximation A' of Eq. (drifta) and the second-order A'' of
    Eq. (drifta2).  The paper's A'' prints "+kappa(lambda_i) + kappa(lambda_l)"
    in its first-order bracket; the expansion (and A' itself) require
    "-kappa(lambda_i) - kappa(lambda_l)", which is what is used here.
  * Black's caplet formula (Section 1) and its implied volatility.
  * The last rate is driftless under the terminal measure (Section 2, remark
    after Eq. (Levy-LIBOR-beta)): its caplet is a European option on an
    exponential NIG variable, priced by Fourier inversion (Lewis 2001) and,
    for time-constant lambda, by direct integration of the NIG density.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.integrate
import scipy.optimize
import scipy.special

from . import quadrature


def nig_gamma(alpha, beta):
    return math.sqrt(alpha * alpha - beta * beta)


def nig_mu(wl):
    if wl.mu is not None:
        return float(wl.mu)
    return -wl.dbar * wl.beta / nig_gamma(wl.alpha, wl.beta)


def kappa(u, alpha, beta, dbar, mu):
    """log E[exp(u H_1)] for NIG(alpha, beta, dbar, mu); complex u allowed
    (principal square root), |Re(u) + beta| < alpha."""
    g = math.sqrt(alpha * alpha - beta * beta)
    u = np.asarray(u)
    root = np.sqrt(alpha * alpha - (beta + u) ** 2)  # principal branch for complex u
    return mu * u + dbar * (g - root)


def kappa_wl(u, wl):
    return kappa(u, wl.alpha, wl.beta, wl.dbar, nig_mu(wl))


def kappa_quad(u, nodes, W):
    """Jump cumulant of the truncated measure as seen by the rule:
    sum_j W_j (e^{u x_j} - 1 - u x_j) / x_j^2."""
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    x = nodes[None, :]
    return (W[None, :] * (np.expm1(u[:, None] * x) - u[:, None] * x) / x ** 2).sum(axis=1)


def kappa_tail(u, alpha, beta, dbar, a):
    """int_{|x|>a} (e^{ux} - 1 - ux) nu(x) dx by adaptive quadrature."""
    f = lambda x: (math.expm1(u * x) - u * x) * float(quadrature.levy_density(x, alpha, beta, dbar))
    right = scipy.integrate.quad(f, a, np.inf, epsabs=1e-15, epsrel=1e-12, limit=400)[0]
    left = scipy.integrate.quad(f, -np.inf, -a, epsabs=1e-15, epsrel=1e-12, limit=400)[0]
    return right + left


# ---------------------------------------------------------------------------
# Drift from the product expansion.
# ---------------------------------------------------------------------------
def drift_jump_exact(i, w, lam, kap):
    """A_i = int [(e^{lam_i x}-1) prod_{l>i} (1 + w_l (e^{lam_l x}-1)) - lam_i x] F(dx)
    via Eq. (product): sum over subsets S of {i+1..n} of prod_{l in S} w_l
    times int (e^{lam_i x}-1) prod_{l in S}(e^{lam_l x}-1) F(dx), each written
    by inclusion-exclusion as sum_{T subset S+{i}} (-1)^{|S|+1-|T|} kappa(lam_T).
    Rates are 1-based: lam[l-1], w[l-1].  ``kap`` is the jump cumulant."""
    n = len(lam)
    later = list(range(i + 1, n + 1))
    total = float(kap(lam[i - 1]))
    for r in range(1, len(later) + 1):
        for S in itertools.combinations(later, r):
            U = (i,) + S
            inner = 0.0
            for t in range(1, len(U) + 1):
                for T in itertools.combinations(U, t):
                    inner += (-1) ** (len(U) - t) * float(kap(sum(lam[m - 1] for m in T)))
            total += np.prod([w[l - 1] for l in S]) * inner
    return total


def drift_jump_first_order(i, w, lam, kap):
    """A' of Eq. (drifta)."""
    n = len(lam)
    li = lam[i - 1]
    out = float(kap(li))
    for l in range(i + 1, n + 1):
        ll = lam[l - 1]
        out += w[l - 1] * (float(kap(li + ll)) - float(kap(li)) - float(kap(ll)))
    return out


def drift_jump_second_order(i, w, lam, kap, printed_signs=False):
    """A'' of Eq. (drifta2).  ``printed_signs=True`` reproduces the first-order
    bracket exactly as printed (+kappa(lam_i) + kappa(lam_l)); the default is
    the inclusion-exclusion reading (-kappa(lam_i) - kappa(lam_l))."""
    n = len(lam)
    li = lam[i - 1]
    out = float(kap(li))
    sgn = 1.0 if printed_signs else -1.0
    for l in range(i + 1, n + 1):
        ll = lam[l - 1]
        out += w[l - 1] * (float(kap(li + ll)) + sgn * float(kap(li)) + sgn * float(kap(ll)))
    for k in range(i + 1, n + 1):
        for l in range(k + 1, n + 1):
            lk, ll = lam[k - 1], lam[l - 1]
            out += w[k - 1] * w[l - 1] * (
                float(kap(li + ll + lk)) - float(kap(li + ll)) - float(kap(li + lk))
                - float(kap(lk + ll)) + float(kap(li)) + float(kap(ll)) + float(kap(lk)))
    return out


# ---------------------------------------------------------------------------
# Black's formula (Section 1).
# ---------------------------------------------------------------------------
def _ncdf(x):
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


def black_caplet(F, K, sigma, T, delta, B_pay):
    """delta B(0, T_{i+1}) [F Phi(d1) - K Phi(d2)]."""
    if K <= 0:
        return delta * B_pay * (F - K)
    if sigma * math.sqrt(T) <= 0:
        return delta * B_pay * max(F - K, 0.0)
    v = sigma * math.sqrt(T)
    d1 = (math.log(F / K) + 0.5 * v * v) / v
    return delta * B_pay * (F * _ncdf(d1) - K * _ncdf(d1 - v))


def black_implied_vol(price, F, K, T, delta, B_pay, lo=1e-6, hi=5.0):
    intrinsic = delta * B_pay * max(F - K, 0.0)
    if price <= intrinsic + 1e-300:
        return float("nan")
    f = lambda s: black_caplet(F, K, s, T, delta, B_pay) - price
    if f(hi) < 0:
        return float("nan")
    return scipy.optimize.brentq(f, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)


# ---------------------------------------------------------------------------
# Last-rate caplet: Fourier inversion and NIG density.
# ---------------------------------------------------------------------------
def nig_pdf(x, alpha, beta, delta, mu):
    g = math.sqrt(alpha * alpha - beta * beta)
    r = np.sqrt(delta * delta + (x - mu) ** 2)
    return alpha * delta / np.pi * scipy.special.k1e(alpha * r) / r * np.exp(
        delta * g + beta * (x - mu) - alpha * r)


def last_caplet_fourier(wl, nodes, W, K):
    """Caplet on L_n fixing at T_n under the log-Euler scheme with the rule's
    compensator kappa_a: L_n(T_n) = L_n(0) exp(sum_k lam_k dH_k - h sum_k
    kappa_a(lam_k)).  Lewis (2001): with forward F and the martingale
    log-return X, E[(F e^X - K)^+] = F - sqrt(FK)/pi int_0^inf
    Re[e^{iu log(F/K)} phi_X(u - i/2)] / (u^2 + 1/4) du."""
    n, s, h = wl.n, wl.s, wl.h
    lam_n = wl.lam[: n * s, n - 1]
    mu = nig_mu(wl)
    kap = lambda z: kappa(z, wl.alpha, wl.beta, wl.dbar, mu)
    ka = kappa_quad(lam_n, nodes, W)
    kex = np.array([float(kap(l)) for l in lam_n])
    F = wl.L0[n] * math.exp(h * np.sum(kex - ka))
    kk = math.log(F / K)

    def phi(u):  # E[exp(i u X)], X martingale log-return
        z = 1j * u
        return np.exp(h * np.sum(kap(z * lam_n + 0j) - z * kex))

    integrand = lambda u: (np.exp(1j * u * kk) * phi(u - 0.5j)).real / (u * u + 0.25)
    val = scipy.integrate.quad(integrand, 0.0, np.inf, epsabs=1e-14, epsrel=1e-12, limit=2000)[0]
    call = F - math.sqrt(F * K) / math.pi * val
    return wl.delta * _bn(wl) * call


def last_caplet_density(wl, nodes, W, K):
    """Same caplet for time-constant lambda_n: X = lam H_T - T kappa_a(lam),
    H_T ~ NIG(alpha, beta, dbar T, mu T); integrate the payoff against the
    NIG density."""
    n = wl.n
    lam = float(wl.lam[0, n - 1])
    T = n * wl.delta
    mu = nig_mu(wl)
    ka = float(kappa_quad(lam, nodes, W)[0])
    L0 = wl.L0[n]
    ystar = (math.log(K / L0) + T * ka) / lam
    f = lambda y: (L0 * math.exp(lam * y - T * ka) - K) * float(
        nig_pdf(y, wl.alpha, wl.beta, wl.dbar * T, mu * T))
    val = scipy.integrate.quad(f, ystar, np.inf, epsabs=1e-15, epsrel=1e-13, limit=2000)[0]
    return wl.delta * _bn(wl) * val


def _bn(wl):
    return float(np.prod(1.0 / (1.0 + wl.delta * np.asarray(wl.L0))))
