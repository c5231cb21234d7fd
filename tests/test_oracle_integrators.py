"""Pins of the oracle's time integration (Eq. cdm, Algorithms 1 and 2, Sec. 2.3)."""
import math

import numpy as np
import pytest

from oracle import eigen, integrators as I
from oracle import integrators as OI
import scipy.linalg as sla
from oracle.basis import gll_points
from oracle.discretization import Discretization, source_vector
from oracle.geometry import Holes


def small(p=2, n=4, physics="scalar", alpha=1e-5, hole=True, stab="none"):
    g = Holes(np.array([[0.5, 0.5, 0.22]])) if hole else None
    return Discretization(2, (n, n), p, physics=physics, geometry=g, alpha=alpha,
                          quad_depth=2, stab=stab, eps=1e-4)


def node_xy(disc):
    xi = gll_points(disc.p)[0]
    lat = disc.lattice_of_node
    g = np.stack([lat % disc.lat[0], lat // disc.lat[0]], axis=1)
    e = np.minimum(g // disc.p, disc.n[None, :] - 1)
    return (e + (xi[g - e * disc.p] + 1.0) / 2.0) * disc.h[None, :]


@pytest.mark.parametrize("physics", ["scalar", "elastic"])
def test_cdm_exact_discrete_mode(physics):
    d = small(physics=physics)
    s = 1.0 / np.sqrt(d.ML)
    lam, Y = np.linalg.eigh(s[:, None] * d.K.toarray() * s[None, :])
    j = len(lam) // 2
    v = s * Y[:, j]
    dt = 0.5 * eigen.dt_crit(lam.max())
    theta = math.acos(1.0 - lam[j] * dt * dt / 2.0)
    for n in (1, 7, 40):
        u, _, _ = I.cdm(d.K, d.ML, dt, n, u0=v)
        np.testing.assert_allclose(u, math.cos(n * theta) * v, atol=1e-11 * np.abs(v).max())


def test_cdm_energy_conserved():
    d = small(p=3)
    rng = np.random.default_rng(1)
    u0 = rng.standard_normal(d.n_dof)
    v0 = rng.standard_normal(d.n_dof)
    dt = 0.8 * eigen.dt_crit(eigen.dense_lambda_max(d.K, d.ML))
    E = []
    for n in range(1, 25):
        u, up, _ = I.cdm(d.K, d.ML, dt, n, u0=u0, v0=v0)
        delta = (u - up) / dt
        E.append(0.5 * delta @ (d.ML * delta) + 0.5 * u @ (d.K @ up))
    E = np.array(E)
    assert np.max(np.abs(E - E[0])) < 1e-12 * abs(E[0])


def test_cdm_continuum_second_order():
    """Unfilled Neumann square, u0 = cos(pi x) cos(pi y): u = cos(sqrt(2) pi t) u0."""
    d = Discretization(2, (4, 4), 6, physics="scalar")
    X = node_xy(d)
    u0 = np.cos(np.pi * X[:, 0]) * np.cos(np.pi * X[:, 1])
    T = 0.4
    errs = []
    for nsteps in (40, 80, 160):
        dt = T / nsteps
        u, _, _ = I.cdm(d.K, d.ML, dt, nsteps, u0=u0)
        errs.append(np.abs(u - math.cos(math.sqrt(2) * np.pi * T) * u0).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4
    # spatial error (spectral) is far below the temporal one at these steps
    u, _, _ = I.cdm(d.K, d.ML, T / 4000, 4000, u0=u0)
    assert np.abs(u - math.cos(math.sqrt(2) * np.pi * T) * u0).max() < 5e-6


@pytest.mark.parametrize("physics", ["scalar", "elastic"])
def test_elementwise_equals_dense_assembly(physics):
    d = small(physics=physics, n=5)
    rng = np.random.default_rng(2)
    u = rng.standard_normal(d.n_dof)
    dense = np.zeros((d.n_dof, d.n_dof))
    for e in d.kept:
        D = d.elem_dofs[e]
        Ke = d.elem_K(e)
        for a in range(len(D)):
            for b in range(len(D)):
                dense[D[a], D[b]] += Ke[a, b]
    np.testing.assert_allclose(d.K.toarray(), dense, atol=1e-13)
    np.testing.assert_allclose(d.apply_K_elementwise(u), dense @ u, atol=1e-12)


def test_imex_equals_cdm_without_cut_cells():
    d = small(hole=False)
    F = d.point_load(np.array([0.3, 0.6]))
    dt = 0.9 * eigen.dt_crit(eigen.dense_lambda_max(d.K, d.ML))
    sys_ = I.ImexSystem(d.K, d.ML, d.consistent_mass(), d.c_dofs(), dt)
    assert len(sys_.c) == 0
    u1, _ = I.imex(sys_, 60, F=F, f_e=5.0)
    u2, _, _ = I.cdm(d.K, d.ML, dt, 60, F=F, f_e=5.0)
    np.testing.assert_allclose(u1, u2, atol=1e-13 * np.abs(u2).max())


def test_imex_all_implicit_is_trapezoidal_newmark():
    d = small()
    F = d.point_load(np.array([0.15, 0.5]))
    M = d.consistent_mass()
    dt = 0.01
    sys_ = I.ImexSystem(d.K, d.ML, M, d.c_dofs(all_dofs=True), dt)
    u1, _ = I.imex(sys_, 50, F=F, f_e=5.0)
    u2, _, _, _ = I.newmark(d.K, M, dt, 50, beta=0.25, gamma=0.5, F=F, f_e=5.0)
    np.testing.assert_allclose(u1, u2, atol=1e-11 * np.abs(u2).max())


def test_imex_stable_where_cdm_is_not():
    d = small(alpha=1e-8, n=6)
    c = d.c_dofs()
    mask = np.ones(d.n_dof, bool)
    mask[c] = False
    s = 1.0 / np.sqrt(d.ML)
    A = (s[:, None] * d.K.toarray() * s[None, :])[np.ix_(mask, mask)]
    lam_d = np.linalg.eigvalsh(A).max()
    lam_full = eigen.dense_lambda_max(d.K, d.ML)
    assert lam_full > 2 * lam_d                 # the lumped cut cells limit CDM
    dt = 0.9 * eigen.dt_crit(lam_d)
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal(d.n_dof) * 1e-3
    sys_ = I.ImexSystem(d.K, d.ML, d.consistent_mass(), c, dt)
    u1, _ = I.imex(sys_, 400, u0=u0)
    with np.errstate(over="ignore", invalid="ignore"):
        u2, _, _ = I.cdm(d.K, d.ML, dt, 400, u0=u0)
    # fictitious-side DOFs carry alpha-scaled mass, so bounded energy allows O(1) amplitudes;
    # the explicit run at the same step overflows
    assert np.isfinite(u1).all() and np.abs(u1).max() < 1e2
    assert (not np.isfinite(u2).all()) or np.abs(u2).max() > 1e8


def test_imex_second_order():
    d = small(n=4, p=2)
    X = node_xy(d)
    u0 = np.cos(np.pi * X[:, 0]) * np.cos(np.pi * X[:, 1])
    T = 0.3
    sol = {}
    for nsteps in (30, 60, 120, 960):
        dt = T / nsteps
        sys_ = I.ImexSystem(d.K, d.ML, d.consistent_mass(), d.c_dofs(), dt)
        sol[nsteps], _ = I.imex(sys_, nsteps, u0=u0)
    e1 = np.abs(sol[30] - sol[960]).max()
    e2 = np.abs(sol[60] - sol[960]).max()
    e3 = np.abs(sol[120] - sol[960]).max()
    assert 3.3 < e1 / e2 < 4.7 and 3.3 < e2 / e3 < 4.7


def test_source_vectors():
    d = small(p=3)
    F = d.point_load(np.array([0.15, 0.5]))
    assert F.sum() == pytest.approx(1.0, rel=1e-13)      # partition of unity, rho = 1
    de = small(p=3, physics="elastic", hole=False)
    Ft = source_vector(de, {"kind": "edge_traction", "y0": 0.4, "y1": 0.6, "t": [1.0, 0.0]})
    assert Ft[0::2].sum() == pytest.approx(0.2, rel=1e-13)
    assert abs(Ft[1::2]).max() == 0.0
    Fp = de.point_load(np.array([0.3, 0.3]), [0.6, 0.8])
    assert Fp[0::2].sum() == pytest.approx(0.6) and Fp[1::2].sum() == pytest.approx(0.8)


def test_observer_interpolation_exact_for_polynomials():
    """Psi(x) = sum_j N_j(x) Psi_j reproduces any field of degree <= p per axis."""
    d = small(p=3, n=4)
    X = node_xy(d)
    f = lambda x, y: 1.0 + 2.0 * x - 3.0 * y + x * y ** 2 + 0.5 * x ** 3 * y ** 3
    u = f(X[:, 0], X[:, 1])
    pts = np.array([[0.13, 0.71], [0.25, 0.25], [0.9, 0.05], [0.0, 1.0]])
    O = d.observer_matrix(pts)
    np.testing.assert_allclose(O @ u, f(pts[:, 0], pts[:, 1]), atol=1e-12)


# ---------------------------------------------------------------- consistent-mass CDM
def _mixed_mass(d):
    """diag(M_L) on the d-DOFs, the consistent block M^cc on the DOFs of cut cells."""
    import scipy.sparse as sp
    c = d.c_dofs()
    Mc = d.consistent_mass().tocsr()
    mask = np.zeros(d.n_dof, bool)
    mask[c] = True
    Dd = sp.diags(np.where(mask, 0.0, d.ML))
    Cc = sp.diags(mask.astype(float)) @ Mc @ sp.diags(mask.astype(float))
    return (Dd + Cc).tocsr(), c


def _direct_consistent_cdm(K, M, dt, steps, F, f_e):
    """u_{k+1} = 2 u_k - u_{k-1} + dt^2 M^{-1} (F_k - K u_k), u_{-1} from v_0 = 0 (Eq. cdm
    with a non-diagonal mass)."""
    import scipy.sparse.linalg as spla
    from oracle.discretization import ricker
    lu = spla.splu(M.tocsc())
    n = K.shape[0]
    u = np.zeros(n)
    up = u + 0.5 * dt * dt * lu.solve(F * ricker(0.0, f_e) - K @ u)
    for k in range(steps):
        un = 2.0 * u - up + dt * dt * lu.solve(F * ricker(k * dt, f_e) - K @ u)
        up, u = u, un
    return u


def test_imex_with_beta_zero_is_the_consistent_mass_cdm():
    from oracle import discretization as OD
    from paper_2501_19013_gb300 import workloads as W
    w = W.plate_holes_imex(n=12, p=2, count=2, seed=3, steps=80).with_(alpha=1e-3)
    d = OD.from_workload(w)
    M, c = _mixed_mass(d)
    lam = sla.eigh(d.K.toarray(), M.toarray(), eigvals_only=True).max()
    dt = 0.9 * 2.0 / math.sqrt(lam)
    F = OD.source_vector(d, w.source)
    sys_ = OI.ImexSystem(d.K, d.ML, d.consistent_mass(), c, dt, beta=0.0)
    u_imex, _ = OI.imex(sys_, w.steps, F=F, f_e=w.f0)
    u_cdm = _direct_consistent_cdm(d.K, M, dt, w.steps, F, w.f0)
    assert np.linalg.norm(u_imex - u_cdm) <= 1e-11 * np.linalg.norm(u_cdm)


def test_consistent_mass_cdm_stability_limit():
    from oracle import discretization as OD
    from paper_2501_19013_gb300 import workloads as W
    w = W.plate_holes_imex(n=10, p=2, count=2, seed=3).with_(alpha=1e-3)
    d = OD.from_workload(w)
    M, c = _mixed_mass(d)
    lam = sla.eigh(d.K.toarray(), M.toarray(), eigvals_only=True).max()
    dtc = 2.0 / math.sqrt(lam)
    rng = np.random.default_rng(0)
    u0 = rng.standard_normal(d.n_dof)
    for f, grows in ((0.99, False), (1.01, True)):
        sys_ = OI.ImexSystem(d.K, d.ML, d.consistent_mass(), c, f * dtc, beta=0.0)
        with np.errstate(all="ignore"):
            u, _ = OI.imex(sys_, 3000, u0=u0)
            nu = np.linalg.norm(u)
        assert (not np.isfinite(nu) or nu > 1e3 * np.linalg.norm(u0)) == grows


def test_threaded_matvec_and_pooled_setup_are_bitwise_serial():
    """The row-blocked threaded mat-vec and the cut-cell integrals on a process pool only
    split the work: a CDM run and the assembled matrices equal the serial ones bitwise."""
    from paper_2501_19013_gb300 import workloads as W
    from oracle.discretization import from_workload
    w = W.plate_holes_elastic(n=12, p=3, count=3, steps=40)
    d1 = from_workload(w)
    d2 = from_workload(w, workers=3)
    assert (d1.K != d2.K).nnz == 0 and np.array_equal(d1.ML, d2.ML)
    F = source_vector(d1, w.source)
    rng = np.random.default_rng(4)
    u0 = rng.standard_normal(d1.n_dof)
    a = OI.cdm(d1.K, d1.ML, 1e-3, 30, u0=u0, F=F, f_e=w.f0)
    b = OI.cdm(d1.K, d1.ML, 1e-3, 30, u0=u0, F=F, f_e=w.f0, threads=5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    l1 = eigen.power_iteration(d1.K, d1.ML, max_iter=50)
    l2 = eigen.power_iteration(d1.K, d1.ML, max_iter=50, threads=4)
    assert l1 == l2


def test_imex_lu_and_cholesky_solvers_agree_when_well_conditioned():
    """Algorithm 2 with S solved by sparse LU or by dense Cholesky: the same scheme, so at
    alpha = 1e-4 (S well conditioned) the two runs agree to rounding."""
    d = small(p=3, n=6, alpha=1e-4)
    c = d.c_dofs()
    dt = 0.5 * eigen.dt_crit(eigen.dense_lambda_max(d.K, d.ML))
    sys_ = OI.ImexSystem(d.K, d.ML, d.consistent_mass(), c, dt)
    rng = np.random.default_rng(2)
    u0 = rng.standard_normal(d.n_dof)
    a, _ = OI.imex(sys_, 40, u0=u0)
    b, _ = OI.imex(sys_, 40, u0=u0, solver="cholesky")
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)
