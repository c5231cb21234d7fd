"""Space-tree quadrature of cut cells (Sec. 1 and Sec. 2.2).

A cut cell is split recursively into 2^d equal children.  A child that the exact box
test finds entirely physical or entirely fictitious becomes a leaf with a constant
indicator (1 or alpha).  A child that is still cut at the maximum depth becomes a leaf
whose indicator alpha^FCM is evaluated at each quadrature point.  Every leaf carries a
tensor Gauss-Legendre rule; the paper says GL points are used in all leaf cells but not
how many -- the reading taken here is p + 1 per direction (exact for the polynomial
integrands of a leaf with constant indicator).

Pins: sum of weights times indicator against the closed-form area of a disk / circular
segment inside a box (error shrinking with depth), exact voxel volumes at depth 1, and
equality with the plain GL rule for uncut cells (tests/test_oracle_quadrature.py); with
depth p + 1, five of the paper's critical time steps of the consistent-mass CDM on the
rotated cube (p = 2, ne = 28 and p = 3, ne = 13; tests/test_timing_table_cpu.py).
"""
from __future__ import annotations

import itertools

import numpy as np

from .basis import gauss_legendre
from .geometry import CUT, OUTSIDE, PHYSICAL


def _tensor_rule(lo, hi, xg, wg):
    d = len(lo)
    pts1 = [lo[k] + (xg + 1.0) * 0.5 * (hi[k] - lo[k]) for k in range(d)]
    w1 = [wg * 0.5 * (hi[k] - lo[k]) for k in range(d)]
    # x fastest
    grids = np.meshgrid(*pts1[::-1], indexing="ij")
    wgrid = np.meshgrid(*w1[::-1], indexing="ij")
    X = np.stack([g.ravel() for g in grids[::-1]], axis=1)
    W = np.prod(np.stack([g.ravel() for g in wgrid], axis=1), axis=1)
    return X, W


def cut_cell_quadrature(geom, lo, hi, p, depth, alpha):
    """Points X (nq, d), weights W (nq,) and indicator values A (nq,) for one cell."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    d = len(lo)
    xg, wg = gauss_legendre(p + 1)
    Xs, Ws, As = [], [], []

    def leaf(l, h, a):
        X, W = _tensor_rule(l, h, xg, wg)
        if a is None:
            A = np.where(geom.in_physical(X), 1.0, alpha)
        else:
            A = np.full(len(W), a)
        Xs.append(X)
        Ws.append(W)
        As.append(A)

    def rec(l, h, level):
        c = geom.classify_box(l, h)
        if c == PHYSICAL:
            leaf(l, h, 1.0)
            return
        if c == OUTSIDE:
            leaf(l, h, alpha)
            return
        if level == depth:
            leaf(l, h, None)
            return
        mid = 0.5 * (l + h)
        for bits in itertools.product((0, 1), repeat=d):
            bits = bits[::-1]  # x fastest
            cl = np.where(np.array(bits) == 0, l, mid)
            ch = np.where(np.array(bits) == 0, mid, h)
            rec(cl, ch, level + 1)

    rec(lo, hi, 0)
    return np.concatenate(Xs), np.concatenate(Ws), np.concatenate(As)


def full_cell_quadrature(lo, hi, p):
    """Plain tensor GL rule with p + 1 points per direction over the whole cell."""
    xg, wg = gauss_legendre(p + 1)
    X, W = _tensor_rule(np.asarray(lo, float), np.asarray(hi, float), xg, wg)
    return X, W, np.ones(len(W))
