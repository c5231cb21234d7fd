"""Full-size checks in the launch configurations the bench times (GPU).

The benchmark workloads are too large for a full oracle run, so one step from a random
state is checked at sampled DOFs against the oracle's local evaluation of Eq. cdm (element
matrices of the cells around each DOF, no assembly), for the FP64 path and for the exact
tensor-core path the bench reports.  The paper's own benchmark (the rotated cube, 13^3
cells, p = 3) is small enough for a full oracle run.

Tolerance of the exact path: the step is u^{k+1} = 2 u^k - u^{k-1} + delta with delta =
dt^2/m (F - K u); 2 u^k - u^{k-1} is exact FP64 on both sides and delta carries one FP32
rounding of the residual (2^-24 relative) plus the digit truncation of u (2^-32 of the
tile's largest value times |K|), so delta is compared at 1e-6 of its largest magnitude.
"""
import numpy as np
import pytest

from helpers import gpu_solver, oracle_disc, rel_l2
from oracle.discretization import ricker, source_vector
from paper_2501_19013_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def sampled_step(w, precision, n_random=40, n_cut=3, seed=11):
    d = oracle_disc(w, assemble=False)
    s = gpu_solver(w, precision)
    assert s.info().n_dof == d.n_dof
    dt = 1e-4
    s.set_dt(dt)
    rng = np.random.default_rng(seed)
    u0 = rng.standard_normal(d.n_dof)
    up = u0 * 0.999
    s.set_state(u0, up, 5)
    s.step(1)
    u1, u0_back = s.get_state()
    s.close()
    assert np.array_equal(u0_back, u0)
    picks = list(rng.choice(d.n_dof, n_random, replace=False))
    for e in d.cut[:: max(1, len(d.cut) // n_cut)][:n_cut]:
        picks += list(d.elem_dofs[e])
    picks = np.array(sorted(set(picks)))
    F = source_vector(d, w.source)
    fk = F[picks] * ricker(5 * dt, w.f0)
    ref = d.local_cdm_update(picks, u0, up, dt, fk=fk)
    base = 2.0 * u0[picks] - up[picks]
    return u1[picks] - base, ref - base, u1[picks], ref


def test_full_size_elastic_plate_exact_sampled_step():
    """256x256 p=4 plane strain, 12 holes, EVS (the bench workload), exact TC kernel."""
    d_g, d_o, _, _ = sampled_step(W.plate_holes_elastic(), "exact")
    assert np.abs(d_g - d_o).max() <= 1e-6 * np.abs(d_o).max()


@pytest.mark.parametrize("precision", ["fp64", "exact"])
def test_full_size_porous_cube_sampled_step(precision):
    """64^3 p=3 porous cube (128^3 voxels, EVS, shared cut matrices): one step at sampled
    DOFs, FP64 to 1e-12 and the exact path at the delta tolerance."""
    d_g, d_o, u_g, u_o = sampled_step(W.porous_voxel(), precision, n_random=30, n_cut=3)
    if precision == "fp64":
        np.testing.assert_allclose(u_g, u_o, rtol=1e-12, atol=1e-12 * np.abs(u_o).max())
    else:
        assert np.abs(d_g - d_o).max() <= 1e-6 * np.abs(d_o).max()


@pytest.fixture(scope="module")
def rotated_cube_oracle():
    from helpers import oracle_cdm
    from oracle import eigen
    w = W.rotated_cube(ne=13, p=2, steps=60)      # quadtree depth p + 1 = 3
    d = oracle_disc(w)
    lam, _ = eigen.power_iteration(d.K, d.ML, max_iter=3000, rtol=1e-10)
    dt = 0.9 * eigen.dt_crit(lam)
    u_o, _, s_o = oracle_cdm(w, d, dt, w.steps)
    return w, d, dt, u_o, s_o


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("exact", 1e-4)])
def test_rotated_cube_full_run(rotated_cube_oracle, precision, tol):
    """The paper's benchmark geometry and load at 13^3 cells, p = 2 (the oracle's set-up of
    p = 3 takes minutes), 60 steps of the full field and the 11 observers against the
    oracle's CDM."""
    w, _, dt, u_o, s_o = rotated_cube_oracle
    s = gpu_solver(w, precision)
    s.set_dt(dt)
    s.set_initial()
    s.step(w.steps)
    s.sync()
    u_g, _ = s.get_state()
    s_g = s.sample(w.steps + 1)
    s.close()
    assert rel_l2(u_g, u_o) <= tol
    assert rel_l2(s_g, s_o) <= tol


def test_rotated_cube_consistent_mass_run(rotated_cube_oracle):
    """The consistent cut mass (Sec. 2.6 with beta = 0) on the benchmark geometry at 13^3
    cells, p = 2: 5 646 c-DOFs and 1.0 M nonzeros in the Cholesky factor of M^cc, whose
    separator rows are long enough that the block solve splits their sums over several CTAs.
    40 steps of the full field and the observers against the oracle's Algorithm 2, and
    bitwise equal on a repeat (the split sums are added in a fixed order).  Tolerance: 1e-10,
    or 30 times the spread of two backward-stable oracle solvers (sparse LU, dense Cholesky)
    where the conditioning of M^cc makes that larger."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    from oracle import discretization as OD, eigen, integrators as OI
    w, d, _, _, _ = rotated_cube_oracle
    w = w.with_(scheme="cdm_consistent", steps=40)
    stab = w.stab == "evs"
    c = d.c_dofs()
    mask = np.zeros(d.n_dof, bool)
    mask[c] = True
    P = sp.diags(mask.astype(float))
    Mc = d.consistent_mass(stabilised=stab).tocsr()
    M = (sp.diags(np.where(mask, 0.0, d.ML)) + P @ Mc @ P).tocsc()
    lam = sla.eigsh(d.K.tocsc(), k=1, M=M, which="LA", return_eigenvectors=False)[0]
    dt = 0.9 * eigen.dt_crit(lam)
    F = OD.source_vector(d, w.source)
    obs = d.observer_matrix(w.observers)
    runs = []
    for solver in ("lu", "cholesky"):
        sys_ = OI.ImexSystem(d.K, d.ML, Mc, c, dt, beta=0.0)
        runs.append(OI.imex(sys_, w.steps, F=F, f_e=w.f0, obs=obs, solver=solver))
    (u_o, s_o), (u_c, s_c) = runs
    tol_u = max(1e-10, 30.0 * rel_l2(u_c, u_o))
    tol_s = max(1e-10, 30.0 * rel_l2(s_c, s_o))
    s = gpu_solver(w, "fp64")
    assert s.info().n_c == len(c)
    s.set_dt(dt)
    s.set_initial()
    s.step(w.steps)
    s.sync()
    u_g, _ = s.get_state()
    s_g = s.sample(w.steps + 1)
    assert rel_l2(u_g, u_o) <= tol_u
    assert rel_l2(s_g, s_o) <= tol_s
    s.set_initial()
    s.step(w.steps)
    s.sync()
    assert np.array_equal(s.get_state()[0], u_g)
    s.close()
