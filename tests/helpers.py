"""Shared helpers of the parity tests: run a workload through the oracle and the library."""
import os

import numpy as np

from oracle import discretization as OD, eigen, integrators as OI
from paper_2501_19013_gb300 import workloads as W


def oracle_disc(w, **kw):
    return OD.from_workload(w, **kw)


def _oracle_cut_parts(args):
    from oracle.quadrature import cut_cell_quadrature
    d, cells = args
    out = {}
    for e in cells:
        lo, hi = d.elem_box(e)
        X, Wq, A = cut_cell_quadrature(d.geom, lo, hi, d.p, d.quad_depth, 0.0)
        out[e] = d._matrices(lo, hi, X, Wq, A) + d._matrices(lo, hi, X, Wq, 1.0 - A)
    return out


def oracle_cut_parts(w, workers=None):
    """The oracle's cut-cell integrals of ``w`` split by the indicator: per cut cell
    (K_phys, M_phys, K_fict, M_fict), the physical and the fictitious part, so that the
    matrices for any alpha are K_phys + alpha K_fict and M_phys + alpha M_fict (the
    integrands are linear in alpha^FCM).  Computed by a pool of spawned processes with the
    oracle's own quadrature and element routines; returns (discretisation without cut
    matrices, parts)."""
    import multiprocessing as mp
    d = OD.from_workload(w, assemble=False)
    n = max(1, min(workers or os.cpu_count() or 1, 8, len(d.cut)))
    chunks = [list(d.cut)[i::n] for i in range(n)]
    parts = {}
    with mp.get_context("spawn").Pool(n) as pool:
        for res in pool.map(_oracle_cut_parts, [(d, c) for c in chunks]):
            parts.update(res)
    return d, parts


def oracle_dt(disc, factor=0.9):
    return factor * eigen.dt_crit(eigen.dense_lambda_max(disc.K, disc.ML))


def oracle_cdm(w, disc, dt, steps, u0=None, v0=None):
    F = OD.source_vector(disc, w.source) if w.source else None
    obs = disc.observer_matrix(w.observers) if w.observers is not None else None
    u, up, samples = OI.cdm(disc.K, disc.ML, dt, steps, u0=u0, v0=v0, F=F, f_e=w.f0, obs=obs)
    return u, up, samples


def gpu_solver(w, precision="fp64", **kw):
    from paper_2501_19013_gb300 import ibfem as ib
    s = ib.from_workload(w, precision=precision, **kw)
    if w.source:
        kind, params = ib.source_params(w)
        s.set_source(kind, params, w.f0)
    if w.observers is not None:
        s.set_observers(w.observers, capacity=max(w.steps, 1))
    return s


def gpu_cdm(w, dt, steps, u0=None, v0=None, precision="fp64"):
    s = gpu_solver(w, precision)
    s.set_dt(dt)
    s.set_initial(u0, v0)
    s.step(steps)
    s.sync()
    u, up = s.get_state()
    samples = s.sample(steps + 1) if w.observers is not None else None
    s.close()
    return u, up, samples


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


SMALL_CASES = {
    "plate_one_hole": lambda: W.plate_one_hole(),
    "elastic_evs": lambda: W.plate_holes_elastic(n=24, p=4, count=3, steps=200),
    "elastic_evs_ragged": lambda: W.plate_holes_elastic(n=19, p=2, count=2, seed=3, steps=150),
    "scalar_mass_scaling": lambda: W.plate_holes_imex(n=30, p=3, count=3, scheme="cdm", steps=200),
    "voxel_3d_evs": lambda: W.porous_voxel(n=6, vn=12, p=3, steps=100),
    "voxel_3d_p2_ragged": lambda: W.porous_voxel(n=7, vn=14, p=2, seed=2, steps=100),
    "rotated_cube_gauss": lambda: W.rotated_cube(ne=6, p=2, quad_depth=2, steps=120),
}
