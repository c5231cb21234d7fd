"""The FP64-grade tensor-core path (IBFEM_EXACT64_TC) against the oracle at the FP64 bar (GPU).

The element contraction runs on the tensor cores as seven exact 8-bit digit slices per
operand with integer node sums; the test holds it to the FP64 path's bounds: the operator
to 1e-13 relative L2 (one apply), the CDM runs of the small cases to 1e-10 after their
configured steps, and the plate benchmark after its 10 000 steps against the oracle's
golden run to 1e-10.
"""
import os

import numpy as np
import pytest

from helpers import SMALL_CASES, gpu_cdm, gpu_solver, oracle_cdm, oracle_disc, oracle_dt, rel_l2
from paper_2501_19013_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "plate_holes_elastic_256_p4.npz")


@pytest.mark.parametrize("case", sorted(SMALL_CASES))
def test_exact64_apply_operator(case):
    w = SMALL_CASES[case]()
    d = oracle_disc(w)
    s = gpu_solver(w, "exact64")
    rng = np.random.default_rng(0)
    for scale in (1.0, 1e-7):
        x = rng.standard_normal(d.n_dof) * scale
        assert rel_l2(s.apply_operator(x), d.K @ x) < 1e-13
    s.close()


@pytest.mark.parametrize("case", sorted(SMALL_CASES))
def test_exact64_cdm_run_matches_oracle(case):
    w = SMALL_CASES[case]()
    d = oracle_disc(w)
    dt = oracle_dt(d)
    u_o, up_o, s_o = oracle_cdm(w, d, dt, w.steps)
    u_g, up_g, s_g = gpu_cdm(w, dt, w.steps, precision="exact64")
    assert rel_l2(u_g, u_o) <= TOL
    assert rel_l2(up_g, up_o) <= TOL
    assert rel_l2(s_g, s_o) <= TOL


def test_exact64_random_state_and_resume():
    """A random initial state (all digit levels busy) and a bitwise resume from a saved state."""
    w = SMALL_CASES["elastic_evs_ragged"]()
    d = oracle_disc(w)
    dt = oracle_dt(d, 0.8)
    rng = np.random.default_rng(4)
    u0 = rng.standard_normal(d.n_dof)
    v0 = rng.standard_normal(d.n_dof)
    u_o, _, _ = oracle_cdm(w, d, dt, 120, u0=u0, v0=v0)
    s = gpu_solver(w, "exact64")
    s.set_dt(dt)
    s.set_initial(u0, v0)
    s.step(60)
    a, b = s.get_state()
    s.step(60)
    u_g, _ = s.get_state()
    assert rel_l2(u_g, u_o) <= TOL
    s.set_state(a, b, 60)
    s.step(60)
    assert np.array_equal(s.get_state()[0], u_g)
    s.close()


def test_exact64_plate_benchmark_after_configured_steps():
    g = dict(np.load(GOLDEN))
    w = W.plate_holes_elastic(steps=int(g["steps"]))
    s = gpu_solver(w, "exact64")
    assert s.info().n_dof == int(g["n_dof"])
    s.set_dt(float(g["dt"]))
    s.set_initial()
    s.step(w.steps)
    s.sync()
    u, up = s.get_state()
    series = s.sample(w.steps + 1)
    s.close()
    idx = g["idx"]
    assert np.abs(u[idx] - g["u"]).max() <= TOL * float(g["u_max"])
    assert np.linalg.norm(u[idx] - g["u"]) <= TOL * np.linalg.norm(g["u"])
    assert abs(np.linalg.norm(u) - float(g["u_norm"])) <= TOL * float(g["u_norm"])
    ref = g["series"]
    got = series[:: int(g["series_every"])]
    assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref)
