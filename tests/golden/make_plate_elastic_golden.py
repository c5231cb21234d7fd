"""Write the oracle's run of the plate benchmark to ``plate_holes_elastic_256_p4.npz``.

The plate benchmark: 2D plane strain (E = 1, nu = 0.3, rho = 1) on the unit plate with 12
seeded holes, 256 x 256 cells of order p = 4, alpha = 1e-12, eigenvalue stabilisation of
the cut cells (eps = 1e-4, f_lambda = 1e-2), a Ricker edge traction (f_e = 10) on x = 0,
y in [0.4, 0.6], dt = 0.9 dt_crit and the configured 10 000 steps of Eq. cdm from rest.

Everything here is the FP64 oracle (``oracle/``), fed by the seeded input generator
(``paper_2501_19013_gb300.workloads``, which holds no solver arithmetic):
* dt_crit by the oracle's power iteration (Sec. 2.3) with the settings the benchmark uses
  for the library (start vector 1 + 0.5 sin(i), at most 2000 products, rtol 1e-7);
* the 10 000 steps by ``oracle.integrators.cdm`` on the assembled stiffness (its mat-vec
  split into row blocks over threads, bitwise the serial product).
Stored: dt, lambda, the iteration count, n_dof, the final field and the one before it at
a seeded sample of DOFs (plus every DOF of eight cut cells), the norms of the full final
fields, and the observer series every 10th step.  Run from the repository root:

    python tests/golden/make_plate_elastic_golden.py [--workers 8] [--steps 10000]

It takes about 20 minutes on 8 cores (set-up about 1 minute, 10 000 mat-vecs).
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plate_holes_elastic_256_p4.npz")
N_SAMPLE = 16384
SERIES_EVERY = 10


def main():
    from oracle import discretization as OD, eigen, integrators as OI
    from paper_2501_19013_gb300 import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--steps", type=int, default=-1)
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args()
    w = W.plate_holes_elastic()
    steps = w.steps if args.steps < 0 else args.steps
    t0 = time.time()
    d = OD.from_workload(w, workers=args.workers)
    print(f"set-up {time.time() - t0:.1f} s: {d.n_dof} DOFs, {len(d.cut)} cut cells", flush=True)
    lam, it = eigen.power_iteration(d.K, d.ML, max_iter=2000, rtol=1e-7, threads=args.workers)
    dt = w.dt_factor * eigen.dt_crit(lam)
    print(f"lambda {lam:.12e} after {it} products, dt {dt:.12e} ({time.time() - t0:.1f} s)", flush=True)
    F = OD.source_vector(d, w.source)
    obs = d.observer_matrix(w.observers)
    u, up, series = OI.cdm(d.K, d.ML, dt, steps, F=F, f_e=w.f0, obs=obs, threads=args.workers)
    print(f"{steps} steps done ({time.time() - t0:.1f} s)", flush=True)
    rng = np.random.default_rng(0x2501_19013)
    idx = set(int(i) for i in rng.choice(d.n_dof, N_SAMPLE, replace=False))
    for e in d.cut[:: max(1, len(d.cut) // 8)][:8]:
        idx.update(int(i) for i in d.elem_dofs[e])
    idx = np.array(sorted(idx), dtype=np.int64)
    np.savez_compressed(args.out, dt=dt, lam=lam, iters=it, n_dof=d.n_dof, steps=steps,
                        idx=idx, u=u[idx], u_prev=up[idx], u_norm=np.linalg.norm(u),
                        u_prev_norm=np.linalg.norm(up), u_max=np.abs(u).max(),
                        series=series[::SERIES_EVERY], series_every=SERIES_EVERY,
                        observers=w.observers, ncomp=d.ncomp)
    print(f"wrote {args.out} ({os.path.getsize(args.out)} bytes)", flush=True)


if __name__ == "__main__":
    main()
