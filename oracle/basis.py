"""1D bases and quadrature rules (Sec. 2.2, "Spatial Discretization").

The spectral cell method uses Lagrange polynomials interpolating the Gauss-Lobatto-
Legendre (GLL) points of order p; the GLL rule also integrates the mass matrix of uncut
cells (nodal lumping, Sec. 2.4) and Gauss-Legendre (GL) points integrate everything else.

Pins (tests/test_oracle_basis.py): textbook GLL nodes/weights for p = 1..4, exactness of
GLL for degree 2p-1 and of GL for degree 2n-1, Lagrange cardinality and partition of unity.
"""
from __future__ import annotations

import numpy as np


def legendre_and_derivative(n: int, x):
    """P_n(x) and P_n'(x) by the three-term recurrence (Bonnet)."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    # derivative from P_n and P_{n-1}: (1 - x^2) P_n' = n (P_{n-1} - x P_n)
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (p0 - x * p1) / (1.0 - x * x)
    # endpoints: P_n'(+-1) = (+-1)^{n+1} n(n+1)/2
    dp = np.where(np.abs(x) == 1.0, np.sign(x) ** (n + 1) * n * (n + 1) / 2.0, dp)
    return p1, dp


def gll_points(p: int):
    """GLL nodes and weights of order p (p + 1 points on [-1, 1]).

    Interior nodes are the roots of P_p'; found by Newton's method on P_p' started from
    the Chebyshev-Gauss-Lobatto points.  Weights w_i = 2 / (p (p + 1) P_p(x_i)^2).
    """
    if p < 1:
        raise ValueError("p >= 1")
    x = -np.cos(np.pi * np.arange(p + 1) / p)
    for _ in range(100):
        # Newton on q(x) = (1 - x^2) P_p'(x), whose roots are exactly the GLL nodes.
        # q'(x) = -p (p + 1) P_p(x) from Legendre's differential equation.
        P, dP = legendre_and_derivative(p, x)
        q = (1.0 - x * x) * dP
        dq = -p * (p + 1) * P
        dx = q / dq
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    x[0], x[-1] = -1.0, 1.0
    P, _ = legendre_and_derivative(p, x)
    w = 2.0 / (p * (p + 1) * P * P)
    return x, w


def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1, 1] (library routine)."""
    return np.polynomial.legendre.leggauss(n)


def lagrange(nodes, x):
    """Values L[a, q] = l_a(x_q) and derivatives D[a, q] = l_a'(x_q).

    Direct product formula: l_a(x) = prod_{b != a} (x - x_b) / (x_a - x_b).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(nodes)
    L = np.ones((m, len(x)))
    D = np.zeros((m, len(x)))
    for a in range(m):
        for b in range(m):
            if b == a:
                continue
            L[a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
        # derivative: sum over the factor that is differentiated
        for c in range(m):
            if c == a:
                continue
            term = np.full(len(x), 1.0 / (nodes[a] - nodes[c]))
            for b in range(m):
                if b == a or b == c:
                    continue
                term = term * (x - nodes[b]) / (nodes[a] - nodes[b])
            D[a] += term
    return L, D
