"""Element matrices of the spectral cell method (Sec. 2.1, 2.2).

Scalar wave (Eq. scalar_wave_equation, weak form Eq. weak_form_extended): with the
indicator alpha^FCM multiplying every integrand,

    K^e_ij = sum_q A_q W_q rho c^2 grad N_i(x_q) . grad N_j(x_q)
    M^e_ij = sum_q A_q W_q rho N_i(x_q) N_j(x_q)

Plane-strain elastodynamics is not in the paper; the textbook operator is used:
K^e = sum_q A_q W_q B^T D B with Lame parameters lambda = E nu / ((1 + nu)(1 - 2 nu)),
mu = E / (2 (1 + nu)) and mass rho N N^T per displacement component.  Local DOFs are
ordered node-major, component-minor; local nodes are lexicographic with x fastest.

The mass of uncut cells uses the GLL rule on the GLL interpolation nodes (nodal lumping,
Sec. 2.4), which gives the diagonal M_ii = rho prod_k w_{a_k} h_k / 2.

Pins: p = 1 closed form, K 1 = 0 (rigid modes for elasticity), symmetry and PSD,
sum of the GLL mass = rho |cell|, cut-path integration of an uncut cell equals the
reference matrix (tests/test_oracle_elements.py).
"""
from __future__ import annotations

import numpy as np

from .basis import gll_points, lagrange


def local_node_exponents(p, d):
    """Array (nn, d) of per-axis node indices a_k, lexicographic with x fastest."""
    m = p + 1
    idx = np.arange(m ** d)
    return np.stack([(idx // m ** k) % m for k in range(d)], axis=1)


def shape_functions(p, lo, hi, X):
    """N (nq, nn) and physical gradients G (nq, d, nn) of the GLL Lagrange basis."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    X = np.atleast_2d(X)
    d = len(lo)
    nodes, _ = gll_points(p)
    h = hi - lo
    xi = 2.0 * (X - lo[None, :]) / h[None, :] - 1.0
    L = []
    D = []
    for k in range(d):
        Lk, Dk = lagrange(nodes, xi[:, k])
        L.append(Lk.T)            # (nq, p+1)
        D.append(Dk.T * (2.0 / h[k]))
    A = local_node_exponents(p, d)
    nq, nn = X.shape[0], A.shape[0]
    N = np.ones((nq, nn))
    G = np.ones((nq, d, nn))
    for k in range(d):
        N *= L[k][:, A[:, k]]
        for j in range(d):
            G[:, j, :] *= (D[k] if j == k else L[k])[:, A[:, k]]
    return N, G


def scalar_matrices(p, lo, hi, X, W, A, rho, c):
    N, G = shape_functions(p, lo, hi, X)
    wa = W * A
    K = rho * c * c * np.einsum("q,qdi,qdj->ij", wa, G, G)
    M = rho * np.einsum("q,qi,qj->ij", wa, N, N)
    return K, M


def lame(E, nu):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def elastic_matrices(p, lo, hi, X, W, A, rho, E, nu):
    """Plane strain, 2D only."""
    N, G = shape_functions(p, lo, hi, X)
    nq, _, nn = G.shape
    B = np.zeros((nq, 3, 2 * nn))
    B[:, 0, 0::2] = G[:, 0, :]
    B[:, 1, 1::2] = G[:, 1, :]
    B[:, 2, 0::2] = G[:, 1, :]
    B[:, 2, 1::2] = G[:, 0, :]
    lam, mu = lame(E, nu)
    Dm = np.array([[lam + 2 * mu, lam, 0.0], [lam, lam + 2 * mu, 0.0], [0.0, 0.0, mu]])
    wa = W * A
    K = np.einsum("q,qai,ab,qbj->ij", wa, B, Dm, B)
    Ms = rho * np.einsum("q,qi,qj->ij", wa, N, N)
    M = np.kron(Ms, np.eye(2))
    return K, M


def gll_mass_diagonal(p, h, rho, ncomp):
    """Diagonal GLL mass of an uncut cell (nodal lumping, Sec. 2.4)."""
    _, w = gll_points(p)
    d = len(h)
    A = local_node_exponents(p, d)
    m = rho * np.prod(np.stack([w[A[:, k]] * h[k] / 2.0 for k in range(d)], axis=1), axis=1)
    return np.repeat(m, ncomp)
