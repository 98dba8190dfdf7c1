"""Gauss rule for the NIG Levy measure, FP64 (oracle side).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the
benchmark).  Independent of the CUDA library's own rule builder.

The drift of Eq. (LIBOR-drift-PT) integrates g(x) = (e^{lambda_i x}-1) prod
beta_l - lambda_i x against the Levy measure F(dx) = nu(x) dx.  Since g is
O(x^2) at the origin, the integral is written against the positive, bounded
weight m(x) = x^2 nu(x) on [-a, a]:

    int g dF ~= sum_j W_j g(x_j) / x_j^2,

where (x_j, W_j) is the Q-point Gauss rule of m.  The paper is silent on the
rule; Section 4 only gives the NIG cumulant.  The NIG Levy density (not printed
in the paper) is the standard one of Barndorff-Nielsen (1997):

    nu(x) = (dbar alpha / pi) e^{beta x} K_1(alpha |x|) / |x|.

Construction (Gautschi's discretised Stieltjes route): discretise m on a
geometrically graded composite Gauss-Legendre mesh, run the Lanczos/Stieltjes
recurrence with full re-orthogonalisation to get the Jacobi matrix, and take
its eigen-decomposition (Golub-Welsch).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.special


def levy_density(x, alpha, beta, dbar):
    """NIG Levy density nu(x), x != 0."""
    ax = np.abs(x)
    return dbar * alpha / np.pi * np.exp(beta * x - alpha * ax) * scipy.special.k1e(alpha * ax) / ax


def x2nu(x, alpha, beta, dbar):
    """m(x) = x^2 nu(x) = (dbar alpha / pi) |x| e^{beta x} K_1(alpha |x|)."""
    ax = np.abs(x)
    return dbar * alpha / np.pi * ax * np.exp(beta * x - alpha * ax) * scipy.special.k1e(alpha * ax)


def _mesh(a, G=32, grade=2.0, smallest=1e-13, outer_panels=16):
    """Composite Gauss-Legendre points and weights on [-a, a], panels graded
    geometrically towards the origin (where m has a log-type kink in its
    second derivative) and uniform further out."""
    t, w = np.polynomial.legendre.leggauss(G)
    edges = [0.0]
    e = smallest * a
    while e < a / outer_panels:
        edges.append(e)
        e *= grade
    edges += list(np.linspace(a / outer_panels, a, outer_panels))
    edges = np.array(edges)
    lo, hi = edges[:-1], edges[1:]
    half = 0.5 * (hi - lo)
    mid = 0.5 * (hi + lo)
    pts = (mid[:, None] + half[:, None] * t[None, :]).ravel()
    wts = (half[:, None] * w[None, :]).ravel()
    return np.concatenate([-pts[::-1], pts]), np.concatenate([wts[::-1], wts])


def discretised_weight(alpha, beta, dbar, a, G=32):
    y, v = _mesh(a, G)
    return y, v * x2nu(y, alpha, beta, dbar)


def jacobi_from_discrete(y, v, Q):
    """Recurrence coefficients of the polynomials orthonormal w.r.t. the
    discrete measure sum_k v_k delta_{y_k} (Lanczos with full
    re-orthogonalisation).  Returns (alpha[Q], beta[Q]) with beta[0] = mass."""
    mu0 = v.sum()
    sv = np.sqrt(v)
    q = [sv / np.sqrt(mu0)]
    al = np.zeros(Q)
    be = np.zeros(Q)
    be[0] = mu0
    prev = np.zeros_like(sv)
    bprev = 0.0
    for k in range(Q):
        al[k] = np.dot(q[k], y * q[k])
        r = y * q[k] - al[k] * q[k] - bprev * prev
        for _ in range(2):
            for qq in q:
                r -= np.dot(qq, r) * qq
        if k + 1 < Q:
            b = np.linalg.norm(r)
            be[k + 1] = b
            prev, bprev = q[k], b
            q.append(r / b)
    return al, be


def gauss_rule(alpha, beta, dbar, a, Q):
    """Q-point Gauss rule of m(x) = x^2 nu(x) on [-a, a]: nodes x_j, weights W_j."""
    y, v = discretised_weight(alpha, beta, dbar, a)
    al, be = jacobi_from_discrete(y, v, Q)
    if Q == 1:
        return np.array([al[0]]), np.array([be[0]])
    lam, vec = scipy.linalg.eigh_tridiagonal(al, be[1:Q])
    W = be[0] * vec[0, :] ** 2
    return lam, W


def rule_for(wl):
    """Nodes and weights for a workload (empty for the Brownian driver)."""
    if wl.driver == "brownian" or wl.Q == 0:
        return np.zeros(0), np.zeros(0)
    return gauss_rule(wl.alpha, wl.beta, wl.dbar, wl.a, wl.Q)
