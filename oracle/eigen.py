"""Critical time step of the CDM (Sec. 2.3): dt_crit = 2 / sqrt(lambda_max(K, M)).

* ``dense_lambda_max``  - LAPACK eigenvalues of M^{-1/2} K M^{-1/2} (tiny grids).
* ``power_iteration``   - the iteration the GPU library runs: w <- A w / ||A w|| on
  A = M^{-1/2} K M^{-1/2}, Rayleigh quotient lambda_k = w^T A w, start vector
  v_i = 1 + 0.5 sin(i) over the DOFs (i = global DOF number), stop when
  |lambda_k - lambda_{k-1}| <= rtol lambda_k or after max_iter products.
  It returns a lower bound of lambda_max (an upper bound of dt_crit).
* ``lanczos_lambda_max``  - the largest eigenvalue of M^{-1/2} K M^{-1/2} by ARPACK's
  Lanczos iteration (scipy), for diagonal M on grids too large for the dense solver.
* ``element_bound``      - max_e lambda_max(K^e, M_L^e), an upper bound of the global
  lambda_max for a diagonal mass assembled from element diagonals.

Pins: power iteration converges to the dense value on tiny grids, the dense value sits
below the element bound, and CDM is stable at 0.99 dt_crit and unstable at 1.01 dt_crit
(tests/test_oracle_eigen.py); the critical steps of the IMEX explicit block on the paper's
rotated cube equal the paper's for p = 2 to 5 (tests/test_oracle_imex_dt_table.py).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from .stabilization import element_lambda_max


def dense_lambda_max(K, ML):
    s = 1.0 / np.sqrt(ML)
    A = s[:, None] * K.toarray() * s[None, :]
    return sla.eigvalsh(A).max()


def lanczos_lambda_max(K, ML):
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    s = 1.0 / np.sqrt(ML)
    A = sp.diags(s) @ K @ sp.diags(s)
    return float(spla.eigsh(A, k=1, which="LA", tol=1e-13, v0=start_vector(A.shape[0]))[0][0])


def start_vector(n):
    return 1.0 + 0.5 * np.sin(np.arange(n, dtype=np.float64))


def power_iteration(K, ML, max_iter=500, rtol=1e-10, mask=None, threads=None):
    """Returns (lambda, iterations).  ``mask`` restricts to a DOF subset (zero elsewhere);
    ``threads`` splits the mat-vec into row blocks (bitwise the serial product)."""
    from .integrators import RowBlockMatvec
    n = K.shape[0]
    Kx = RowBlockMatvec(K, threads)
    s = 1.0 / np.sqrt(ML)
    w = start_vector(n)
    if mask is not None:
        w = np.where(mask, w, 0.0)
    w = w / np.linalg.norm(w)
    lam_old = None
    lam = 0.0
    it = 0
    for it in range(1, max_iter + 1):
        z = s * Kx(s * w)
        if mask is not None:
            z = np.where(mask, z, 0.0)
        lam = float(w @ z)
        nz = np.linalg.norm(z)
        w = z / nz
        if lam_old is not None and abs(lam - lam_old) <= rtol * abs(lam):
            break
        lam_old = lam
    Kx.close()
    return lam, it


def element_bound(disc):
    lam = 0.0
    for e in disc.kept:
        lam = max(lam, element_lambda_max(disc.elem_K(e), disc.elem_ml(e)))
    return lam


def dt_crit(lam):
    return 2.0 / math.sqrt(lam)
