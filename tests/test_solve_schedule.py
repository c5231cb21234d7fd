"""The schedule of the GPU block triangular solves, checked on the host (no GPU).

The c-set solve of Algorithm 2 (Sec. 2.6) and of the consistent-mass CDM runs on the GPU
as two dependency-driven sweeps over the supernodes of a nested-dissection order: each
CTA waits only on the supernodes linked to its own by edges of the elimination tree, in a
ticket order that must be topological, and splits long rows over CTAs.
``ibfem_check_solve_schedule`` factors S on the host and replays both sweeps over random
asynchronous orders of ready supernodes, with rows not yet final set to NaN: a wait the
schedule misses shows up as a counted violation (and a NaN), a wrong block or split as an
error against plain substitution.
"""
import pytest

from paper_2501_19013_gb300 import ibfem as ib
from paper_2501_19013_gb300 import workloads as W

CASES = {
    "imex_plate_p3": (lambda: W.plate_holes_imex(n=40, p=3, count=3, seed=1, steps=10), "imex", 0.25 * 1e-6),
    "imex_plate_p3_alpha1e-4": (lambda: W.plate_holes_imex(n=40, p=3, count=3, seed=1, steps=10).with_(alpha=1e-4),
                                "imex", 0.25 * 4e-6),
    "consistent_plate_p2": (lambda: W.plate_holes_imex(n=27, p=2, count=2, seed=5, steps=10).with_(
        alpha=1e-4, stab="none"), "cdm_consistent", 0.0),
    "consistent_voxel_3d": (lambda: W.porous_voxel(n=6, vn=12, p=2, steps=10), "cdm_consistent", 0.0),
    # the paper's geometry at p = 2: separators long enough that rows are split over CTAs
    "consistent_rotated_cube_p2": (lambda: W.rotated_cube(ne=13, p=2, steps=10), "cdm_consistent", 0.0),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_schedule_is_sound_and_matches_substitution(case):
    make, scheme, beta_dt2 = CASES[case]
    s = ib.from_workload(make(), precision="fp64", host_only=True, scheme=scheme)
    assert s.info().n_c > 0
    for seed in (0, 1, 2):
        violations, err = s.check_solve_schedule(beta_dt2, seed=seed)
        assert violations == 0
        assert err <= 1e-12
    s.close()


def test_schedule_check_errors():
    w = W.plate_holes_imex(n=27, p=2, count=2, seed=5, steps=10).with_(alpha=1e-4)
    s = ib.from_workload(w, precision="fp64", host_only=True, scheme="imex")
    with pytest.raises(ib.IbfemError) as e:
        s.check_solve_schedule(-1.0)
    assert e.value.code == ib.ERR_ARG
    s.close()
    c = ib.from_workload(w.with_(scheme="cdm"), precision="fp64", host_only=True, scheme="cdm")
    with pytest.raises(ib.IbfemError) as e:
        c.check_solve_schedule(0.0)
    assert e.value.code == ib.ERR_STATE
    c.close()
