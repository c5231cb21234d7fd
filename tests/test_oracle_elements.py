"""Pins of the oracle's element matrices (Sec. 2.2, Eq. weak_form_extended)."""
import numpy as np
import pytest

from oracle import elements as el
from oracle.discretization import Discretization
from oracle.geometry import Holes
from oracle.quadrature import cut_cell_quadrature, full_cell_quadrature


def ref(p, d, h=0.5, physics="scalar"):
    lo = np.zeros(d)
    hi = np.full(d, h)
    X, W, A = full_cell_quadrature(lo, hi, p)
    if physics == "scalar":
        return el.scalar_matrices(p, lo, hi, X, W, A, 1.0, 1.0)
    return el.elastic_matrices(p, lo, hi, X, W, A, 1.0, 1.0, 0.3)


def test_bilinear_closed_form():
    # textbook bilinear square: K = 1/6 [[4,-1,-1,-2],...], M = h^2/36 [[4,2,2,1],...]
    K, M = ref(1, 2, h=0.3)
    Kx = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    Mx = 0.3 ** 2 / 36.0 * np.array([[4, 2, 2, 1], [2, 4, 1, 2], [2, 1, 4, 2], [1, 2, 2, 4]])
    np.testing.assert_allclose(K, Kx, atol=1e-14)
    np.testing.assert_allclose(M, Mx, atol=1e-15)
    np.testing.assert_allclose(el.gll_mass_diagonal(1, np.array([0.3, 0.3]), 1.0, 1), 0.3 ** 2 / 4)


@pytest.mark.parametrize("p,d", [(2, 2), (3, 2), (4, 2), (2, 3), (3, 3)])
def test_scalar_reference_properties(p, d):
    K, M = ref(p, d)
    np.testing.assert_allclose(K, K.T, atol=1e-13)
    assert np.abs(K @ np.ones(len(K))).max() < 1e-12
    ev = np.linalg.eigvalsh(K)
    assert ev[0] > -1e-12 and ev[1] > 1e-6      # PSD with a one-dimensional null space
    m = el.gll_mass_diagonal(p, np.full(d, 0.5), 1.0, 1)
    assert m.sum() == pytest.approx(0.5 ** d, rel=1e-14)
    assert M.sum() == pytest.approx(0.5 ** d, rel=1e-13)


@pytest.mark.parametrize("p", [1, 2, 4])
def test_elastic_rigid_modes(p):
    K, M = ref(p, 2, physics="elastic")
    np.testing.assert_allclose(K, K.T, atol=1e-13)
    A = el.local_node_exponents(p, 2)
    from oracle.basis import gll_points
    x = (gll_points(p)[0][A] + 1) * 0.25     # node coordinates in [0, 0.5]^2
    tx = np.zeros(2 * len(A)); tx[0::2] = 1
    ty = np.zeros(2 * len(A)); ty[1::2] = 1
    rot = np.zeros(2 * len(A)); rot[0::2] = -x[:, 1]; rot[1::2] = x[:, 0]
    for v in (tx, ty, rot):
        assert np.abs(K @ v).max() < 1e-12
    ev = np.linalg.eigvalsh(K)
    assert ev[2] < 1e-12 and ev[3] > 1e-6       # exactly three rigid modes


@pytest.mark.parametrize("physics,p", [("scalar", 2), ("scalar", 4), ("elastic", 2), ("elastic", 4)])
def test_patch_test_linear_field(physics, p):
    """Assembled K of an uncut grid times a linear field vanishes at interior nodes and
    the energy equals area * strain^T D strain (pins B, D and the assembly)."""
    disc = Discretization(2, (3, 3), p, physics=physics)
    from oracle.basis import gll_points
    xi = gll_points(p)[0]
    lat = disc.lattice_of_node
    g = np.stack([lat % disc.lat[0], lat // disc.lat[0]], axis=1)
    e = np.minimum(g // p, disc.n[None, :] - 1)
    X = (e + (xi[g - e * p] + 1.0) / 2.0) * disc.h[None, :]   # GLL node coordinates
    a, b, c, d = 0.3, -0.7, 0.5, 0.2
    if physics == "scalar":
        u = a * X[:, 0] + b * X[:, 1]
        energy = a * a + b * b
    else:
        u = np.zeros(disc.n_dof)
        u[0::2] = a * X[:, 0] + b * X[:, 1]
        u[1::2] = c * X[:, 0] + d * X[:, 1]
        lam, mu = el.lame(1.0, 0.3)
        eps = np.array([a, d, b + c])
        Dm = np.array([[lam + 2 * mu, lam, 0], [lam, lam + 2 * mu, 0], [0, 0, mu]])
        energy = eps @ Dm @ eps
    Ku = disc.K @ u
    interior = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    mask = np.repeat(interior, disc.ncomp)
    assert np.abs(Ku[mask]).max() < 1e-11
    assert u @ Ku == pytest.approx(energy, rel=1e-12)


def test_cut_path_reproduces_reference_and_alpha():
    p = 3
    h = 0.25
    K_ref, M_ref = ref(p, 2, h=h)
    far = Holes(np.array([[5.0, 5.0, 0.1]]))
    X, W, A = cut_cell_quadrature(far, [0, 0], [h, h], p, 3, 1e-5)
    K, M = el.scalar_matrices(p, [0, 0], [h, h], X, W, A, 1.0, 1.0)
    np.testing.assert_allclose(K, K_ref, atol=1e-14)
    # a cell inside a hole: every integrand carries alpha
    inside = Holes(np.array([[0.1, 0.1, 1.0]]))
    X, W, A = cut_cell_quadrature(inside, [0, 0], [h, h], p, 3, 1e-5)
    K, M = el.scalar_matrices(p, [0, 0], [h, h], X, W, A, 1.0, 1.0)
    np.testing.assert_allclose(M, 1e-5 * M_ref, rtol=1e-12, atol=1e-20)
    np.testing.assert_allclose(K, 1e-5 * K_ref, rtol=1e-12, atol=1e-18)
