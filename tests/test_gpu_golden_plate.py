"""The plate benchmark after its configured step count against the FP64 oracle (GPU).

``tests/golden/plate_holes_elastic_256_p4.npz`` holds the oracle's run of the benchmark
workload (256 x 256 cells, p = 4 plane strain, 12 holes, EVS, edge traction, 10 000 steps
at 0.9 dt_crit from rest), written by ``tests/golden/make_plate_elastic_golden.py``, which
calls only the oracle.  The library runs the same steps with the stored dt in the launch
configuration the bench times (the exact kernel with its autotuned tile) and is compared
element by element at the stored DOF sample, by the norm of the full field, and on the
observer series.

Tolerances: the FP64 path at 1e-10 (relative to the field's largest magnitude, element by
element, and relative L2), the exact tensor-core path at 1e-4, the bar of mixed precision.
"""
import os

import numpy as np
import pytest

from helpers import gpu_solver
from paper_2501_19013_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "plate_holes_elastic_256_p4.npz")


@pytest.fixture(scope="module")
def golden():
    if not os.path.exists(GOLDEN):
        pytest.fail("missing golden file; write it with tests/golden/make_plate_elastic_golden.py")
    return dict(np.load(GOLDEN))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("exact", 1e-4)])
def test_plate_benchmark_after_configured_steps(golden, precision, tol):
    g = golden
    w = W.plate_holes_elastic(steps=int(g["steps"]))
    s = gpu_solver(w, precision)
    assert s.info().n_dof == int(g["n_dof"])
    if precision == "exact":
        s.autotune(reps=3)
    s.set_dt(float(g["dt"]))
    s.set_initial()
    s.step(w.steps)
    s.sync()
    u, up = s.get_state()
    series = s.sample(w.steps + 1)
    s.close()
    idx = g["idx"]
    scale = float(g["u_max"])
    assert scale > 0.0
    err = np.abs(u[idx] - g["u"])
    assert err.max() <= tol * scale, f"max |du| / max|u| = {err.max() / scale:.3e}"
    assert np.linalg.norm(u[idx] - g["u"]) <= tol * np.linalg.norm(g["u"])
    assert np.abs(up[idx] - g["u_prev"]).max() <= tol * scale
    assert abs(np.linalg.norm(u) - float(g["u_norm"])) <= tol * float(g["u_norm"])
    ref = g["series"]
    got = series[:: int(g["series_every"])]
    assert got.shape == ref.shape
    nc = int(g["ncomp"])
    for o in range(ref.shape[1] // nc):
        cols = slice(o * nc, (o + 1) * nc)
        nr = np.linalg.norm(ref[:, cols])
        assert nr > 0.0, "every observer of the benchmark is reached by the wave"
        assert np.linalg.norm(got[:, cols] - ref[:, cols]) <= tol * nr
