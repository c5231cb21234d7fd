"""Pins of the critical time step (Sec. 2.3: dt_crit = 2 / sqrt(lambda_max))."""
import numpy as np
import pytest

from oracle import eigen, integrators as I
from oracle.discretization import Discretization
from oracle.geometry import Holes


@pytest.mark.parametrize("physics", ["scalar", "elastic"])
def test_dense_below_element_bound_and_power_converges(physics):
    g = Holes(np.array([[0.43, 0.55, 0.21]]))   # asymmetric: isolated top eigenvalue
    d = Discretization(2, (5, 5), 2, physics=physics, geometry=g, alpha=1e-6, quad_depth=3)
    lam = eigen.dense_lambda_max(d.K, d.ML)
    assert lam <= eigen.element_bound(d) * (1 + 1e-12)
    lp, it = eigen.power_iteration(d.K, d.ML, max_iter=5000, rtol=1e-14)
    assert lp <= lam * (1 + 1e-12)
    assert lp == pytest.approx(lam, rel=1e-9)


def test_stability_limit():
    g = Holes(np.array([[0.43, 0.55, 0.21]]))
    d = Discretization(2, (5, 5), 2, geometry=g, alpha=1e-4, quad_depth=2)
    lam = eigen.dense_lambda_max(d.K, d.ML)
    rng = np.random.default_rng(0)
    u0 = rng.standard_normal(d.n_dof)
    u_ok, _, _ = I.cdm(d.K, d.ML, 0.99 * eigen.dt_crit(lam), 400, u0=u0)
    u_bad, _, _ = I.cdm(d.K, d.ML, 1.01 * eigen.dt_crit(lam), 400, u0=u0)
    assert np.abs(u_ok).max() < 50 * np.abs(u0).max()
    assert np.abs(u_bad).max() > 1e6 * np.abs(u0).max()
