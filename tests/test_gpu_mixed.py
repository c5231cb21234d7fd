"""Mixed-precision tensor-core path (tcgen05, TF32 operands, FP64 state) against the oracle.

The element contractions run in TF32 on the tensor cores (three passes hi*hi + hi*lo +
lo*hi for about FP32 accuracy, or one pass); the state and the central-difference update
stay FP64.  The bar for a mixed variant to count is a relative L2 error <= 1e-4 against the
FP64 oracle after the configured steps.
"""
import numpy as np
import pytest

from helpers import SMALL_CASES, gpu_cdm, gpu_solver, oracle_cdm, oracle_disc, oracle_dt, rel_l2

pytestmark = pytest.mark.gpu

MIXED_BAR = 1e-4
TC_CASES = ["plate_one_hole", "elastic_evs", "elastic_evs_ragged", "scalar_mass_scaling",
            "voxel_3d_evs", "voxel_3d_p2_ragged"]
# relative error of one operator application K x for a random x
APPLY_TOL = {"tf32x3": 2e-6, "tf32": 5e-3}


@pytest.mark.parametrize("prec", ["tf32x3", "tf32"])
@pytest.mark.parametrize("case", TC_CASES)
def test_tc_apply_operator(case, prec):
    w = SMALL_CASES[case]()
    d = oracle_disc(w)
    s = gpu_solver(w, precision=prec)
    x = np.random.default_rng(0).standard_normal(d.n_dof)
    y = s.apply_operator(x)
    assert rel_l2(y, d.K @ x) < APPLY_TOL[prec]
    s.close()


@pytest.mark.parametrize("case", TC_CASES)
def test_tc_cdm_run_within_mixed_bar(case):
    w = SMALL_CASES[case]()
    d = oracle_disc(w)
    dt = oracle_dt(d)
    u_o, up_o, s_o = oracle_cdm(w, d, dt, w.steps)
    u_g, up_g, s_g = gpu_cdm(w, dt, w.steps, precision="tf32x3")
    assert rel_l2(u_g, u_o) <= MIXED_BAR
    # observer series: error relative to the field amplitude (an observer the wave has not
    # reached sees only an exponentially small precursor, whose relative error is noise)
    assert np.abs(s_g - s_o).max() <= MIXED_BAR * np.abs(u_o).max()


def test_tc_step_counter_and_ring_follow_the_fp64_path():
    """Same step bookkeeping as the FP64 path: rows of the observer ring, resume."""
    w = SMALL_CASES["plate_one_hole"]()
    d = oracle_disc(w)
    dt = oracle_dt(d)
    a = gpu_solver(w, precision="tf32x3")
    a.set_dt(dt)
    a.set_initial()
    a.step(77)
    rows = a.sample(1000)
    assert rows.shape[0] == 78
    assert a.info().step == 77
    a.close()
