"""The paper's critical time steps of the consistent-mass CDM on the rotated cube (golden
values in tests/golden/timing_table_cpu_dt_crit.txt: p = 2, ne = 28 and p = 3, ne = 13),
on the CPU.

The oracle's discretisation (its cut cells integrated in a process pool, split into the
physical and the fictitious part so that one integration per grid serves every alpha)
gives the alpha-stabilised rows (eps = 0) and the eigenvalue-stabilised row (Sec. 2.5); the
library's host setup (element stiffnesses and consistent element masses through
``ibfem_get_element_mass``) gives the eigenvalue-stabilised row.  Each assembles K and the
consistent mass M (GLL diagonal in uncut cells, Sec. 2.4); the largest eigenvalue of
M^{-1} K comes from ARPACK, and dt_crit = 2 / sqrt(lambda_max) (Sec. 2.3).

These pin the oracle's classification, space-tree quadrature, alpha^FCM, consistent mass
and eigenvalue stabilisation to the paper's own numbers; the last row fixes the reading of
the scale of M^s (M^f the GLL mass of a full cell: five digits; the exactly integrated full
mass misses the row by 3 %)."""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import discretization as OD
from oracle.stabilization import evs, hrz
from paper_2501_19013_gb300 import workloads as W

ib = pytest.importorskip("paper_2501_19013_gb300.ibfem")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "timing_table_cpu_dt_crit.txt")


def rows():
    out = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            p, ne, a, eps, dt = line.split()
            out.append((int(p), int(ne), float(a), float(eps), float(dt) * 1e-3))
    return out


def grids():
    return sorted({(p, ne) for p, ne, _, _, _ in rows()})


def cube(p, ne, alpha, eps):
    return W.rotated_cube(ne=ne, p=p, alpha=alpha, stab="evs" if eps > 0 else "none", eps=eps,
                          quad_depth=p + 1)


def dt_crit(K, M):
    lu = spla.splu(M.tocsc())
    op = spla.LinearOperator(K.shape, matvec=lambda x: lu.solve(K @ x))
    lam = spla.eigs(op, k=1, which="LR", tol=1e-12, v0=np.ones(K.shape[0]), maxiter=50000)[0][0].real
    return 2.0 / np.sqrt(lam)


@pytest.fixture(scope="module", params=grids(), ids=lambda g: f"p{g[0]}_ne{g[1]}")
def oracle_parts(request):
    from helpers import oracle_cut_parts
    p, ne = request.param
    d, parts = oracle_cut_parts(cube(p, ne, 1e-8, 0.0))
    return p, ne, d, parts


def test_oracle_dt_crit_matches_the_paper(oracle_parts):
    p, ne, d, parts = oracle_parts
    assert d.f_lambda == 1e-2
    for alpha, eps, dt_paper in [r[2:] for r in rows() if r[:2] == (p, ne)]:
        d.eps, d.stab, d.alpha = eps, ("evs" if eps > 0 else "none"), alpha
        for e, (Kp, Mp, Kf, Mf) in parts.items():
            Mo = Mp + alpha * Mf
            Ms = evs(Mo, d.M_full, eps, d.f_lambda) if eps > 0 else Mo
            d.K_cut[e], d.M_cut_cons[e], d.M_cut_stab[e] = Kp + alpha * Kf, Mo, Ms
            d.ml_cut[e], d.scale_cut[e] = hrz(Ms), 1.0
        d._assemble()
        dt = dt_crit(d.K, d.consistent_mass(stabilised=True))
        assert abs(dt - dt_paper) <= 2e-4 * dt_paper, (p, ne, alpha, eps, dt, dt_paper)   # four digits


def test_oracle_split_integrals_equal_the_direct_ones(oracle_parts):
    """K_phys + alpha K_fict equals the oracle's direct integration at that alpha."""
    p, ne, d, parts = oracle_parts
    w = cube(p, ne, 1e-4, 0.0)
    dd = OD.from_workload(w, assemble=False)
    for e in list(parts)[:: max(1, len(parts) // 8)]:
        dd._cut_matrices(e)
        Kp, Mp, Kf, Mf = parts[e]
        np.testing.assert_allclose(Kp + 1e-4 * Kf, dd.K_cut[e], rtol=1e-12, atol=1e-12 * np.abs(dd.K_cut[e]).max())
        np.testing.assert_allclose(Mp + 1e-4 * Mf, dd.M_cut_cons[e], rtol=1e-12,
                                   atol=1e-12 * np.abs(dd.M_cut_cons[e]).max())


def assembled(s, d):
    """Global K and consistent M (kept-DOF order of the oracle's numbering, which the
    library shares) from the library's element matrices."""
    nl = d.n_loc
    ii, jj = np.meshgrid(np.arange(nl), np.arange(nl), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    Kref, _ = s.element(d.uncut[0])
    Mref = s.element_mass(d.uncut[0])
    uncut = set(d.uncut)
    rk, ck, vk, vm = [], [], [], []
    for e in list(d.uncut) + list(d.cut):
        K, M = (Kref, Mref) if e in uncut else (s.element(e)[0], s.element_mass(e))
        D = d.elem_dofs[e]
        rk.append(D[ii]), ck.append(D[jj]), vk.append(K.ravel()), vm.append(M.ravel())
    n = d.n_dof
    r, c = np.concatenate(rk), np.concatenate(ck)
    return (sp.csr_matrix((np.concatenate(vk), (r, c)), shape=(n, n)),
            sp.csr_matrix((np.concatenate(vm), (r, c)), shape=(n, n)))


@pytest.mark.parametrize("p,ne,alpha,eps,dt_paper", [r for r in rows() if r[3] > 0])
def test_host_setup_evs_dt_crit_matches_the_paper(p, ne, alpha, eps, dt_paper):
    w = cube(p, ne, alpha, eps)
    s = ib.from_workload(w, host_only=True, scheme="cdm_consistent")
    d = OD.from_workload(w, assemble=False)      # classes and DOF numbering only
    assert s.info().n_dof == d.n_dof
    K, M = assembled(s, d)
    s.close()
    dt = dt_crit(K, M)
    assert abs(dt - dt_paper) <= 2e-4 * dt_paper   # four significant digits
