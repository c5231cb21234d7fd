"""GPU parity of the FP64 path against the oracle (calls through the C ABI)."""
import numpy as np
import pytest

from helpers import SMALL_CASES, gpu_cdm, gpu_solver, oracle_cdm, oracle_disc, oracle_dt, rel_l2
from oracle import eigen
from paper_2501_19013_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# FP64 parity bound: relative L2 <= 1e-10 against the oracle after the configured steps
TOL = 1e-10


@pytest.mark.parametrize("case", sorted(SMALL_CASES))
def test_apply_operator(case):
    w = SMALL_CASES[case]()
    d = oracle_disc(w)
    s = gpu_solver(w)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(d.n_dof)
    y = s.apply_operator(x)
    ref = d.K @ x
    assert rel_l2(y, ref) < 1e-13
    np.testing.assert_allclose(s.lumped_mass(), d.ML, rtol=1e-9)
    s.close()


@pytest.mark.parametrize("case", sorted(SMALL_CASES))
def test_cdm_run_matches_oracle(case):
    w = SMALL_CASES[case]()
    d = oracle_disc(w)
    dt = oracle_dt(d)
    steps = w.steps
    u_o, up_o, s_o = oracle_cdm(w, d, dt, steps)
    u_g, up_g, s_g = gpu_cdm(w, dt, steps)
    assert rel_l2(u_g, u_o) <= TOL
    assert rel_l2(up_g, up_o) <= TOL
    assert s_g.shape == s_o.shape
    assert rel_l2(s_g, s_o) <= TOL


def test_cdm_random_initial_state():
    w = SMALL_CASES["elastic_evs_ragged"]()
    d = oracle_disc(w)
    dt = oracle_dt(d, 0.8)
    rng = np.random.default_rng(4)
    u0 = rng.standard_normal(d.n_dof)
    v0 = rng.standard_normal(d.n_dof)
    u_o, _, _ = oracle_cdm(w, d, dt, 120, u0=u0, v0=v0)
    u_g, _, _ = gpu_cdm(w, dt, 120, u0=u0, v0=v0)
    assert rel_l2(u_g, u_o) <= TOL


@pytest.mark.parametrize("case", ["plate_one_hole", "elastic_evs", "voxel_3d_evs"])
def test_power_iteration_matches_oracle(case):
    w = SMALL_CASES[case]()
    d = oracle_disc(w)
    # rtol < 0 never triggers the stopping rule: exactly 60 products on both sides
    lam_o, it_o = eigen.power_iteration(d.K, d.ML, max_iter=60, rtol=-1.0)
    s = gpu_solver(w)
    dt, lam_g, it_g = s.crit_dt(max_iter=60, rtol=-1.0)
    assert it_g == it_o == 60
    assert lam_g == pytest.approx(lam_o, rel=1e-11)
    assert dt == pytest.approx(2.0 / np.sqrt(lam_o), rel=1e-11)
    # with the stopping rule the iteration count matches too
    lam_o2, it_o2 = eigen.power_iteration(d.K, d.ML, max_iter=3000, rtol=1e-7)
    _, lam_g2, it_g2 = s.crit_dt(max_iter=3000, rtol=1e-7)
    assert abs(it_g2 - it_o2) <= 1
    assert lam_g2 == pytest.approx(lam_o2, rel=1e-9)
    s.close()


def test_resume_is_bitwise():
    w = SMALL_CASES["plate_one_hole"]()
    d = oracle_disc(w)
    dt = oracle_dt(d)
    a = gpu_solver(w)
    a.set_dt(dt)
    a.set_initial()
    a.step(70)
    u_full, up_full = None, None
    b = gpu_solver(w)
    b.set_dt(dt)
    b.set_initial()
    b.step(33)
    u_mid, up_mid = b.get_state()
    c = gpu_solver(w)
    c.set_dt(dt)
    c.set_state(u_mid, up_mid, 33)
    c.step(37)
    u_full, up_full = a.get_state()
    u_res, up_res = c.get_state()
    assert np.array_equal(u_full, u_res) and np.array_equal(up_full, up_res)
    for s in (a, b, c):
        s.close()


def test_divergence_is_reported():
    from paper_2501_19013_gb300 import ibfem as ib
    w = SMALL_CASES["plate_one_hole"]()
    d = oracle_disc(w)
    lam = eigen.dense_lambda_max(d.K, d.ML)
    s = gpu_solver(w)
    s.set_dt(1.5 * eigen.dt_crit(lam))
    rng = np.random.default_rng(1)
    s.set_initial(rng.standard_normal(d.n_dof))
    s.step(4000)
    with pytest.raises(ib.IbfemError) as ei:
        s.sync()
    assert ei.value.code == ib.ERR_DIVERGED
    s.close()


def test_full_size_elastic_plate_sampled_step():
    """256x256 p=4 plane strain, 12 holes, EVS: one GPU step from a random state checked
    at sampled DOFs (uncut interior, cut-cell and traction-edge nodes) against the oracle's
    local evaluation of Eq. cdm from element matrices (no assembly)."""
    w = W.plate_holes_elastic()
    d = oracle_disc(w, assemble=False)
    s = gpu_solver(w)
    assert s.info().n_dof == d.n_dof
    dt = 1e-4
    s.set_dt(dt)
    rng = np.random.default_rng(7)
    u0 = rng.standard_normal(d.n_dof)
    s.set_state(u0, u0 * 0.999, 5)
    s.step(1)
    u1, u0_back = s.get_state()
    assert np.array_equal(u0_back, u0)
    # sampled DOFs: random ones plus every DOF of three cut cells
    picks = list(rng.choice(d.n_dof, 40, replace=False))
    for e in d.cut[:: max(1, len(d.cut) // 3)][:3]:
        picks += list(d.elem_dofs[e])
    picks = np.array(sorted(set(picks)))
    from oracle.discretization import ricker, source_vector
    F = source_vector(d, w.source)
    fk = F[picks] * ricker(5 * dt, w.f0)
    ref = d.local_cdm_update(picks, u0, u0 * 0.999, dt, fk=fk)
    np.testing.assert_allclose(u1[picks], ref, rtol=1e-12, atol=1e-12 * np.abs(u0).max())
    s.close()
