"""Pins of eigenvalue stabilisation, HRZ lumping and mass scaling (Sec. 2.4, 2.5)."""
import numpy as np
import pytest

from oracle import eigen
from oracle.discretization import Discretization
from oracle.geometry import Holes
from oracle.stabilization import element_lambda_max, evs, hrz


def badly_cut(physics="scalar", stab="none", eps=0.0, p=3):
    g = Holes(np.array([[0.5, 0.5, 0.2]]))
    return Discretization(2, (8, 8), p, physics=physics, geometry=g, alpha=1e-8,
                          quad_depth=3, stab=stab, eps=eps, f_lambda=1e-2)


@pytest.mark.parametrize("physics", ["scalar", "elastic"])
def test_evs_structure(physics):
    d = badly_cut(physics, "evs", 1e-4)
    hit = 0
    for e in d.cut:
        Mo, Me = d.M_cut_cons[e], d.M_cut_stab[e]
        Ms = (Me - Mo) / 1e-4
        if np.abs(Ms).max() == 0:
            continue
        hit += 1
        np.testing.assert_allclose(Ms, Ms.T, atol=1e-13)
        # M^s = s P with P the projector onto the small-eigenvalue eigenspace of M^o
        s = Ms.max() / 1.0
        assert Ms.max() == pytest.approx(d.M_full.max(), rel=1e-10)
        P = Ms / (d.M_full.max() / (Ms / Ms.max() * 1.0).max())
        lam = np.linalg.eigvalsh(Ms)
        assert lam.min() > -1e-10 * lam.max()
        # idempotence of the unscaled projector
        Pn = Ms / Ms.max()
        Pn = Pn / np.max(np.linalg.eigvalsh(Pn))
        np.testing.assert_allclose(Pn @ Pn, Pn, atol=1e-10)
        # projector range = eigenvectors of M^o below f_lambda * lambda_max
        lo, V = np.linalg.eigh(Mo)
        small = lo < 1e-2 * lo.max()
        np.testing.assert_allclose(Pn, V[:, small] @ V[:, small].T, atol=1e-8)
    assert hit > 0


def test_evs_invariant_to_eigenvector_sign_and_basis():
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    lam = np.array([1e-9, 1e-9, 1e-6, 0.5, 0.7, 1.0])     # a degenerate small cluster
    Mo = Q @ np.diag(lam) @ Q.T
    Mf = np.eye(6) * 0.3 + 0.01
    a = evs(Mo, Mf, 1e-4, 1e-2)
    # rotate inside the degenerate cluster and flip signs: same result
    R = np.eye(6)
    c, s = np.cos(0.7), np.sin(0.7)
    R[:2, :2] = [[c, -s], [s, c]]
    R[2, 2] = -1
    Q2 = Q @ R
    b = evs(Q2 @ np.diag(lam) @ Q2.T, Mf, 1e-4, 1e-2)
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_hrz_preserves_mass_and_positivity():
    d = badly_cut("scalar", "none")
    for e in d.cut:
        ml = d.ml_cut[e]
        assert np.all(ml > 0)
        assert ml.sum() == pytest.approx(d.M_cut_cons[e].sum(), rel=1e-12)
    total = sum(d.elem_ml(e).sum() for e in d.kept)
    assert d.ML.sum() == pytest.approx(total, rel=1e-12)
    assert np.all(d.ML > 0)
    # HRZ of a diagonal matrix is the identity map
    D = np.diag([1.0, 2.0, 3.0])
    np.testing.assert_allclose(hrz(D), [1, 2, 3])


def test_mass_scaling_bounds_lambda():
    d = badly_cut("scalar", "mass_scaling", p=2)
    for e in d.cut:
        assert element_lambda_max(d.K_cut[e], d.ml_cut[e]) <= d.lam_ref * (1 + 1e-10)
    lam = eigen.dense_lambda_max(d.K, d.ML)
    assert lam <= d.lam_ref * (1 + 1e-10)
    # without scaling the badly cut cells raise lambda far above the uncut value
    d0 = badly_cut("scalar", "none", p=2)
    assert eigen.dense_lambda_max(d0.K, d0.ML) > 1.5 * d.lam_ref


def test_evs_raises_critical_step():
    d0 = badly_cut("scalar", "none", p=2)
    d1 = badly_cut("scalar", "evs", 1e-4, p=2)
    assert eigen.dense_lambda_max(d1.K, d1.ML) < eigen.dense_lambda_max(d0.K, d0.ML)
