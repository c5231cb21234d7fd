"""Classification of cells against the physical domain (Sec. 2.2 and Sec. 3.1).

The extended domain is a Cartesian box meshed by a uniform grid.  The indicator
alpha^FCM is 1 in the physical domain Omega and alpha in the fictitious part
(Eq. weak_form_extended).  A cell is

* ``OUTSIDE``  - entirely fictitious; such cells are dropped from the discretisation
  (Sec. 3.2, selection procedure: "elements completely outside" are removed),
* ``CUT``      - intersected by the immersed boundary (space-tree quadrature),
* ``PHYSICAL`` - entirely inside Omega (uncut: GLL mass, shared reference stiffness).

Three geometry descriptions are supported:

* holes:  circles (2D) / spheres (3D) of fictitious material in the unit box,
* voxels: an image with 1 = void (fictitious), 0 = solid, spanning the extended box,
* rotated box: the physical domain is a cube of edge ``l_p`` rotated about the centre of
  the extended cube (the paper's benchmark, Sec. 3.1).

Readings of the paper where it is silent: tangency (distance == r) counts as not cut;
a box covered by the union of two holes but by neither alone is classified CUT (its
quadrature then resolves alpha pointwise).

Pins: brute-force point sampling of boxes (tests/test_oracle_geometry.py) and the exact
DOF counts of Table 3 for the rotated cube.
"""
from __future__ import annotations

import math

import numpy as np

OUTSIDE, CUT, PHYSICAL = 0, 1, 2


class Holes:
    """Fictitious circular / spherical holes: rows (centre..., r)."""

    def __init__(self, holes):
        h = np.asarray(holes, dtype=np.float64)
        self.h = h.reshape(len(h), -1)

    def classify_box(self, lo, hi):
        lo = np.asarray(lo, dtype=np.float64)
        hi = np.asarray(hi, dtype=np.float64)
        d = len(lo)
        any_cut = False
        for row in self.h:
            c, r = row[:d], row[d]
            dmin2 = 0.0
            dmax2 = 0.0
            for k in range(d):
                gap = max(lo[k] - c[k], 0.0, c[k] - hi[k])
                dmin2 += gap * gap
                far = max(abs(c[k] - lo[k]), abs(c[k] - hi[k]))
                dmax2 += far * far
            if dmax2 <= r * r:
                return OUTSIDE          # box inside this hole
            if dmin2 < r * r:
                any_cut = True          # boundary of this hole crosses the box
        return CUT if any_cut else PHYSICAL

    def in_physical(self, x):
        """Boolean per point: True if the point lies in Omega (outside every hole)."""
        x = np.atleast_2d(np.asarray(x, dtype=np.float64))
        d = x.shape[1]
        inside_any = np.zeros(len(x), dtype=bool)
        for row in self.h:
            c, r = row[:d], row[d]
            inside_any |= np.sum((x - c[None, :]) ** 2, axis=1) < r * r
        return ~inside_any


class Voxels:
    """Voxel image (1 = void) spanning the extended box ``[lo, hi]``.

    Array index order is reversed coordinates: img[y, x] in 2D, img[z, y, x] in 3D.
    """

    def __init__(self, img, lo, hi):
        self.img = np.asarray(img, dtype=np.uint8)
        self.d = self.img.ndim
        self.vn = np.array(self.img.shape[::-1])  # voxels per coordinate axis (x, y[, z])
        self.lo = np.asarray(lo, dtype=np.float64)[: self.d]
        self.hi = np.asarray(hi, dtype=np.float64)[: self.d]

    def _range(self, lo, hi):
        rel0 = (np.asarray(lo) - self.lo) / (self.hi - self.lo) * self.vn
        rel1 = (np.asarray(hi) - self.lo) / (self.hi - self.lo) * self.vn
        i0 = np.floor(rel0 + 1e-9).astype(int)
        i1 = np.ceil(rel1 - 1e-9).astype(int)
        i0 = np.clip(i0, 0, self.vn - 1)
        i1 = np.clip(i1, i0 + 1, self.vn)
        return i0, i1

    def classify_box(self, lo, hi):
        i0, i1 = self._range(lo, hi)
        sl = tuple(slice(i0[k], i1[k]) for k in reversed(range(self.d)))
        block = self.img[sl]
        if np.all(block == 1):
            return OUTSIDE
        if np.all(block == 0):
            return PHYSICAL
        return CUT

    def in_physical(self, x):
        x = np.atleast_2d(np.asarray(x, dtype=np.float64))
        rel = (x - self.lo[None, :]) / (self.hi - self.lo)[None, :] * self.vn[None, :]
        idx = np.clip(np.floor(rel).astype(int), 0, self.vn[None, :] - 1)
        return self.img[tuple(idx[:, k] for k in reversed(range(self.d)))] == 0


def cardan_matrix(phi, theta, psi, order="xyz"):
    """Rotation matrix from Cardan angles (radians); ``order`` names the axis sequence
    of the intrinsic rotations (R = R_a(phi) R_b(theta) R_c(psi))."""
    def R(axis, a):
        c, s = math.cos(a), math.sin(a)
        if axis == "x":
            return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
        if axis == "y":
            return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
        return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
    return R(order[0], phi) @ R(order[1], theta) @ R(order[2], psi)


class RotatedBox:
    """Physical domain = cube of edge ``lp`` centred at ``centre``, axes = columns of T.

    x = centre + T x' maps the cube's local frame (Sec. 3.1, "x = T x'")."""

    def __init__(self, lp, centre, T):
        self.half = lp / 2.0
        self.c = np.asarray(centre, dtype=np.float64)
        self.T = np.asarray(T, dtype=np.float64)

    def classify_box(self, lo, hi):
        lo = np.asarray(lo, dtype=np.float64)
        hi = np.asarray(hi, dtype=np.float64)
        cb = 0.5 * (lo + hi)
        hb = 0.5 * (hi - lo)
        # separating axis test between the axis-aligned box and the rotated cube
        axes = [np.eye(3)[k] for k in range(3)] + [self.T[:, k] for k in range(3)]
        for i in range(3):
            for j in range(3):
                ax = np.cross(np.eye(3)[i], self.T[:, j])
                if np.linalg.norm(ax) > 1e-12:
                    axes.append(ax / np.linalg.norm(ax))
        dc = self.c - cb
        for L in axes:
            rb = np.sum(hb * np.abs(L))
            rc = self.half * np.sum(np.abs(self.T.T @ L))
            if abs(dc @ L) >= rb + rc:
                return OUTSIDE
        # all 8 corners inside the cube -> physical
        corners = np.array([[lo[0] if a == 0 else hi[0], lo[1] if b == 0 else hi[1],
                             lo[2] if c == 0 else hi[2]]
                            for a in (0, 1) for b in (0, 1) for c in (0, 1)])
        if np.all(self.in_physical(corners)):
            return PHYSICAL
        return CUT

    def in_physical(self, x):
        x = np.atleast_2d(np.asarray(x, dtype=np.float64))
        loc = (x - self.c[None, :]) @ self.T  # x' = T^T (x - c)
        return np.all(np.abs(loc) <= self.half, axis=1)


def make_geometry(dim, holes=None, voxels=None, lo=None, hi=None, rotated_box=None):
    if rotated_box is not None:
        rb = np.asarray(rotated_box, dtype=np.float64)
        return RotatedBox(rb[0], rb[1:4], rb[4:13].reshape(3, 3))
    if voxels is not None:
        return Voxels(voxels, lo, hi)
    if holes is not None and len(holes) > 0:
        return Holes(np.asarray(holes, dtype=np.float64).reshape(-1, dim + 1))
    return None
