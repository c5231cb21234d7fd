"""Pins of the space-tree quadrature (Sec. 1, 2.2) against exact areas/volumes."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle.geometry import Holes, Voxels
from oracle.quadrature import cut_cell_quadrature, full_cell_quadrature


def disk_box_area(cx, cy, r, x0, x1, y0, y1):
    """Area of disk(c, r) intersected with [x0,x1]x[y0,y1] by adaptive 1D integration of
    the clipped chord length (independent of any space tree)."""
    a, b = max(x0, cx - r), min(x1, cx + r)
    if b <= a:
        return 0.0

    def chord(x):
        s = math.sqrt(max(r * r - (x - cx) ** 2, 0.0))
        return max(0.0, min(y1, cy + s) - max(y0, cy - s))

    pts = [a, b]
    for yy in (y0, y1):
        dy = yy - cy
        if abs(dy) < r:
            s = math.sqrt(r * r - dy * dy)
            pts += [cx - s, cx + s]
    pts = sorted(p for p in pts if a <= p <= b)
    total = 0.0
    for lo, hi in zip(pts[:-1], pts[1:]):
        if hi > lo:
            total += quad(chord, lo, hi, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    return total


@pytest.mark.parametrize("box", [(0.4, 0.5, 0.3, 0.4), (0.55, 0.7, 0.55, 0.7), (0.2, 0.45, 0.45, 0.6)])
def test_physical_area_converges(box):
    cx, cy, r = 0.5, 0.5, 0.2
    x0, x1, y0, y1 = box
    g = Holes(np.array([[cx, cy, r]]))
    exact_phys = (x1 - x0) * (y1 - y0) - disk_box_area(cx, cy, r, x0, x1, y0, y1)
    errs = []
    for depth in (1, 3, 5, 7):
        X, W, A = cut_cell_quadrature(g, [x0, y0], [x1, y1], 3, depth, alpha=0.0)
        errs.append(abs(np.sum(W * A) - exact_phys))
    area = (x1 - x0) * (y1 - y0)
    assert errs[-1] < 2e-4 * area
    assert errs[3] < errs[0]
    # integral of the constant 1 (alpha = 1) is exact regardless of the tree
    X, W, A = cut_cell_quadrature(g, [x0, y0], [x1, y1], 3, 4, alpha=1.0)
    assert np.sum(W * A) == pytest.approx(area, rel=1e-13)


def test_voxel_depth1_exact():
    # 2 voxels per element and direction: depth 1 leaves coincide with voxels
    rng = np.random.default_rng(3)
    img = (rng.random((8, 8, 8)) < 0.4).astype(np.uint8)
    g = Voxels(img, [0, 0, 0], [1, 1, 1])
    alpha = 1e-3
    for e in [(0, 0, 0), (1, 2, 3), (3, 3, 3)]:
        lo = np.array(e) * 0.25
        hi = lo + 0.25
        X, W, A = cut_cell_quadrature(g, lo, hi, 3, 1, alpha)
        sub = img[2 * e[2]:2 * e[2] + 2, 2 * e[1]:2 * e[1] + 2, 2 * e[0]:2 * e[0] + 2]
        v = 0.125 ** 3
        exact = v * (np.sum(sub == 0) + alpha * np.sum(sub == 1))
        assert np.sum(W * A) == pytest.approx(exact, rel=1e-13)


def test_uncut_cell_matches_full_rule():
    g = Holes(np.array([[5.0, 5.0, 0.1]]))
    X, W, A = cut_cell_quadrature(g, [0, 0], [0.25, 0.25], 4, 3, 1e-5)
    Xf, Wf, Af = full_cell_quadrature([0, 0], [0.25, 0.25], 4)
    np.testing.assert_allclose(X, Xf)
    np.testing.assert_allclose(W, Wf)
    np.testing.assert_allclose(A, 1.0)
