"""The oracle's volumetric Gaussian load (Sec. 3.1, load term of Eq. weak_form_extended)
against closed forms: the integral of the Gaussian (partition of unity: sum_i F_i =
int f_s), its centre (linear completeness: sum_i x_i F_i = x_l int f_s) and the half-space
case (the physical cube's face through the centre of the Gaussian, with the fictitious
half dropped as outside cells)."""
import math

import numpy as np

from oracle import elements as el
from oracle.basis import gll_points
from oracle.discretization import Discretization
from oracle.geometry import RotatedBox


def node_coordinates(d):
    X = np.zeros((d.n_nodes, d.dim))
    xi, _ = gll_points(d.p)
    A = el.local_node_exponents(d.p, d.dim)
    for e in d.kept:
        lo, hi = d.elem_box(e)
        x = lo[None, :] + (xi[A] + 1.0) * 0.5 * (hi - lo)[None, :]
        X[d.node_of_lattice[d.elem_lat[e]]] = x
    return X


def test_gauss_load_integral_and_centre_2d():
    d = Discretization(2, (10, 10), 3, geometry=None, rho=1.7)
    xl, sig = np.array([0.47, 0.52]), 0.03
    F = d.gauss_load(xl, sig)
    total = 1.7 * 2.0 * math.pi * sig * sig
    assert abs(F.sum() - total) <= 1e-11 * total
    X = node_coordinates(d)
    np.testing.assert_allclose(X.T @ F, xl * total, rtol=1e-11)


def test_gauss_load_narrow_relative_to_cells_3d():
    # sigma = h / 5 as in the benchmark (h = 0.05, sigma = 0.01)
    d = Discretization(3, (6, 6, 6), 2, geometry=None, lo=(0, 0, 0), hi=(0.3, 0.3, 0.3))
    xl, sig = np.array([0.151, 0.148, 0.155]), 0.01
    F = d.gauss_load(xl, sig)
    total = (2.0 * math.pi) ** 1.5 * sig ** 3
    assert abs(F.sum() - total) <= 1e-10 * total
    X = node_coordinates(d)
    np.testing.assert_allclose(X.T @ F, xl * total, rtol=1e-10)


def test_gauss_load_on_a_face_counts_the_physical_half():
    # unrotated cube [0.3, 0.7]^3 on a 10^3 grid: its face x = 0.3 is a cell boundary, the
    # cells left of it are outside (dropped), so exactly half the Gaussian remains
    box = RotatedBox(0.4, [0.5, 0.5, 0.5], np.eye(3))
    d = Discretization(3, (10, 10, 10), 2, geometry=box, alpha=1e-12, quad_depth=1,
                       lo=(0, 0, 0), hi=(1, 1, 1), assemble=False)
    xl, sig = np.array([0.3, 0.5, 0.5]), 0.02
    F = d.gauss_load(xl, sig)
    total = 0.5 * (2.0 * math.pi) ** 1.5 * sig ** 3
    assert abs(F.sum() - total) <= 1e-10 * total


def test_gauss_load_weights_the_fictitious_part_by_alpha():
    # face x = 0.32 inside the cells [0.3, 0.4] (on a subcell boundary: m = 5 subcells of
    # 0.02); the cut cells keep the slab 0.30 < x < 0.32 with weight alpha
    alpha = 0.3
    box = RotatedBox(0.36, [0.5, 0.5, 0.5], np.eye(3))
    d = Discretization(3, (10, 10, 10), 2, geometry=box, alpha=alpha, quad_depth=1,
                       lo=(0, 0, 0), hi=(1, 1, 1), assemble=False)
    xl, sig = np.array([0.32, 0.5, 0.5]), 0.02
    F = d.gauss_load(xl, sig)
    full = (2.0 * math.pi) ** 1.5 * sig ** 3
    slab = 0.5 * math.erf(1.0 / math.sqrt(2.0))      # mass of the Gaussian in [x_l - sigma, x_l]
    total = full * (0.5 + alpha * slab)
    assert abs(F.sum() - total) <= 1e-10 * total
