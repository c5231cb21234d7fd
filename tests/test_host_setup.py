"""Host-side discretisation of the library against the oracle (no GPU needed: the
library is created with host_only=1, which runs the C++ setup and no device code)."""
import math
import os

import numpy as np
import pytest

from oracle import discretization as OD
from oracle.geometry import Holes, Voxels
from paper_2501_19013_gb300 import workloads as W

ib = pytest.importorskip("paper_2501_19013_gb300.ibfem")
if not os.path.exists(ib.LIB_PATH):
    pytest.skip("libibfem.so not built", allow_module_level=True)


def compare(w, rtol=1e-11):
    d = OD.from_workload(w)
    s = ib.from_workload(w, host_only=True)
    inf = s.info()
    assert inf.n_dof == d.n_dof
    assert inf.n_cut == len(d.cut) and inf.n_uncut == len(d.uncut)
    np.testing.assert_array_equal(s.cut_cells(), d.cut)
    ml = s.lumped_mass()
    np.testing.assert_allclose(ml, d.ML, rtol=rtol, atol=0)
    Kr, mr = s.element(d.uncut[0])
    np.testing.assert_allclose(Kr, d.K_ref, rtol=rtol, atol=rtol * np.abs(d.K_ref).max())
    np.testing.assert_allclose(mr, d.m_gll, rtol=rtol)
    for e in d.cut[:: max(1, len(d.cut) // 25)]:
        K, m = s.element(e)
        np.testing.assert_allclose(K, d.K_cut[e], rtol=rtol, atol=rtol * np.abs(d.K_cut[e]).max())
        np.testing.assert_allclose(m, d.ml_cut[e], rtol=1e-9, atol=1e-9 * m.max())
    assert inf.lambda_ref == pytest.approx(d.lam_ref, rel=1e-11)
    s.close()


def test_plate_one_hole_setup():
    compare(W.plate_one_hole())


def test_elastic_evs_setup():
    compare(W.plate_holes_elastic(n=24, p=4, count=3, steps=10))


def test_mass_scaling_setup():
    compare(W.plate_holes_imex(n=20, p=3, count=2, scheme="cdm"))


def test_voxel_3d_evs_setup():
    compare(W.porous_voxel(n=6, vn=12, p=2, steps=10))


@pytest.mark.parametrize("p,ne,dofs", [(4, 9, 21109), (5, 7, 22706)])
def test_rotated_cube_dofs_table3(p, ne, dofs):
    """Library classifier + numbering reproduce the Table 3 DOF counts (Sec. 3.1)."""
    from oracle.geometry import cardan_matrix
    a = math.radians(10.0)
    T = cardan_matrix(a, a, a, "zyx")
    rb = np.concatenate([[0.3, 0.25, 0.25, 0.25], T.ravel()])
    s = ib.Solver(3, (ne, ne, ne), p, lo=(0, 0, 0), hi=(0.5, 0.5, 0.5), rotated_box=rb,
                  quad_depth=0, host_only=True)
    assert s.info().n_dof == dofs


def test_imex_partition_size():
    """c-set = DOFs with support in a cut cell (Sec. 2.6)."""
    w = W.plate_holes_imex(n=30, p=3, count=3, seed=2)
    d = OD.from_workload(w)
    s = ib.from_workload(w, host_only=True)
    assert s.info().n_c == len(d.c_dofs())
    s.close()


def test_voxel_blocks_share_cut_matrices():
    # cut cells with equal voxel blocks (2 voxels per cell and axis) share one matrix set;
    # every cut cell's shared set must equal the oracle's own integration of that cell
    w = W.porous_voxel(n=8, vn=16, p=2, steps=10)
    d = OD.from_workload(w)
    s = ib.from_workload(w, host_only=True)
    inf = s.info()
    assert inf.n_cut_matrices < inf.n_cut
    for e in d.cut:
        K, m = s.element(e)
        np.testing.assert_allclose(K, d.K_cut[e], rtol=1e-11, atol=1e-11 * np.abs(d.K_cut[e]).max())
        np.testing.assert_allclose(m, d.ml_cut[e], rtol=1e-9, atol=1e-9 * m.max())
    s.close()
    h = ib.from_workload(W.plate_one_hole(), host_only=True)
    assert h.info().n_cut_matrices == h.info().n_cut   # curved boundaries: no sharing
    h.close()


def test_rotated_cube_workload_geometry():
    """The benchmark's load centre lies on the cube face x' = -l/2 (Sec. 3.1), and every
    observer lies in a kept cell (the oracle's classification)."""
    from oracle.geometry import RotatedBox
    w = W.rotated_cube(ne=6, p=2)
    rb = w.rotated_box
    T = rb[4:13].reshape(3, 3)
    c = rb[1:4]
    xl = np.asarray(w.source["x"])
    loc = T.T @ (xl - c)
    assert abs(loc[0] + rb[0] / 2) < 1e-12 and abs(loc[1]) < 1e-12 and abs(loc[2]) < 1e-12
    d = OD.from_workload(w, assemble=False)
    for x in w.observers:
        d.locate(x)        # raises if the point is in no kept cell
    box = RotatedBox(rb[0], c, T)
    assert box.in_physical(w.observers).all()


def test_clone_needs_a_device_handle():
    """ibfem_clone shares device arrays, so it refuses a host-only source (STATE) and a
    null source (ARG) before touching the device."""
    import ctypes as C
    h = ib.from_workload(W.plate_one_hole(), host_only=True)
    with pytest.raises(ib.IbfemError) as ei:
        h.clone()
    assert ei.value.code == ib.ERR_STATE
    out = C.c_void_p()
    assert ib.lib().ibfem_clone(None, C.byref(out)) == ib.ERR_ARG
    assert h.info().shared_device_bytes == 0
    h.close()


def test_element_mass_of_the_consistent_schemes():
    """ibfem_get_element_mass: the cut cells' consistent mass M^o + eps M^s (Eq.
    epsilon_stabilization) as the oracle integrates and stabilises it, the GLL diagonal
    for uncut cells; a lumped-mass CDM handle keeps no consistent cut mass (STATE)."""
    w = W.plate_holes_imex(n=20, p=3, count=3, seed=2).with_(scheme="cdm_consistent", stab="evs",
                                                              eps=1e-4, f_lambda=1e-2)
    d = OD.from_workload(w)
    s = ib.from_workload(w, host_only=True)
    for e in d.cut:
        M = s.element_mass(e)
        Mo = d.M_cut_stab[e]
        np.testing.assert_allclose(M, Mo, rtol=1e-10, atol=1e-10 * np.abs(Mo).max())
        assert not np.allclose(M, d.M_cut_cons[e])      # the stabilisation is in
    e = d.uncut[0]
    np.testing.assert_allclose(s.element_mass(e), np.diag(d.m_gll), rtol=1e-14)
    s.close()
    h = ib.from_workload(w.with_(scheme="cdm"), host_only=True)
    with pytest.raises(ib.IbfemError) as ei:
        h.element_mass(d.cut[0])
    assert ei.value.code == ib.ERR_STATE
    np.testing.assert_allclose(h.element_mass(e), np.diag(d.m_gll), rtol=1e-14)
    h.close()
