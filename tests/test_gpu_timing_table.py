"""The paper's critical time steps of the consistent-mass CDM on the rotated cube (golden
values in tests/golden/timing_table_dt_crit.txt) through the library's power iteration on
M^{-1} K with the consistent cut mass (GPU)."""
import os

import pytest

from paper_2501_19013_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "timing_table_dt_crit.txt")


def rows():
    out = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            p, ne, a, dt = line.split()
            out.append((int(p), int(ne), float(a), float(dt) * 1e-3))
    return out


@pytest.mark.parametrize("p,ne,alpha,dt_paper", rows())
def test_consistent_mass_dt_crit_matches_the_paper(p, ne, alpha, dt_paper):
    from paper_2501_19013_gb300 import ibfem as ib
    w = W.rotated_cube(ne=ne, p=p, alpha=alpha, stab="none", eps=0.0, quad_depth=p + 1)
    s = ib.from_workload(w, scheme="cdm_consistent")
    dt, lam, it = s.crit_dt(max_iter=3000, rtol=1e-9)
    s.close()
    assert abs(dt - dt_paper) <= 2e-4 * dt_paper   # four significant digits
