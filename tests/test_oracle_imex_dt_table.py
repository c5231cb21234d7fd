"""The paper's critical time steps of the IMEX scheme on the rotated cube (golden values in
tests/golden/timing_table_imex_dt_crit.txt) from the oracle: the explicit block of the
partition (Sec. 2.6: DOFs without support in a cut cell, uncut reference stiffness and GLL
mass, Sec. 2.2 and 2.4) and dt_crit = 2 / sqrt(lambda_max) (Sec. 2.3).

This pins the oracle's classification of the rotated cube (Sec. 3.1), its DOF numbering,
the c-set definition, K_ref and the GLL mass for p = 2 to 5 against the paper's numbers."""
import os

import pytest

from oracle import discretization as OD, eigen
from paper_2501_19013_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "timing_table_imex_dt_crit.txt")


def rows():
    out = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            p, ne, dt = line.split()
            out.append((int(p), int(ne), float(dt) * 1e-3))
    return out


@pytest.mark.parametrize("p,ne,dt_paper", rows())
def test_imex_explicit_block_dt_crit_matches_the_paper(p, ne, dt_paper):
    w = W.rotated_cube(ne=ne, p=p, alpha=1e-12, stab="none", eps=0.0)
    d = OD.from_workload(w, assemble=False)
    K, ml, _ = d.explicit_block()
    dt = eigen.dt_crit(eigen.lanczos_lambda_max(K, ml))
    assert abs(dt - dt_paper) <= 2e-4 * dt_paper     # four significant digits
