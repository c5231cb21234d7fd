"""Time integration (Sec. 2.3 and Sec. 2.6).

* ``cdm``    - central differences with the lumped mass, Eq. cdm:
               Psi_{k+1} = 2 Psi_k - Psi_{k-1} + dt^2 M^{-1} (F_k - K Psi_k).
               Start-up (the paper is silent): Psi_{-1} = Psi_0 - dt Psi'_0 +
               dt^2 / 2 M^{-1} (F_0 - K Psi_0), i.e. Algorithm 1 with beta = 0.
* ``newmark`` - the predictor-corrector of Algorithm 1 (general beta, gamma) with a sparse
               direct solve of S = M + beta dt^2 K.
* ``imex``   - Newmark IMEX of Algorithm 2: CDM on the d-DOFs (support only in uncut cells,
               diagonal M^dd), trapezoidal Newmark (beta = 1/4, gamma = 1/2) on the c-DOFs
               (support in a cut cell, consistent M^cc).  The initial d history uses the
               same start-up as ``cdm``; Algorithm 1 and 2 write F_k in their
               initialisation line, read as F_0.

All loops are plain; K is the assembled sparse matrix (library mat-vec as a step).
Samples: row k of the returned series is the observer reading of Psi_k, k = 0..nsteps.
``threads`` splits the mat-vec K u into row blocks taken by a thread pool (scipy releases
the interpreter lock in its CSR product); each row's sum is the serial one, so the result
is bitwise the same for any thread count.

Pins: exact discrete modal solution and energy conservation of CDM, temporal rate,
IMEX == CDM without cut cells, IMEX == trapezoidal Newmark with all DOFs implicit,
IMEX stable at the uncut-grid step where CDM blows up (tests/test_oracle_integrators.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .discretization import ricker


class RowBlockMatvec:
    """y = K x with the rows of the CSR matrix K split into ``threads`` contiguous blocks,
    each multiplied by scipy on a pool thread; threads <= 1 is the plain product."""

    def __init__(self, K, threads=None):
        self.K = K.tocsr()
        self.threads = int(threads or 1)
        self.pool = None
        if self.threads > 1:
            from concurrent.futures import ThreadPoolExecutor
            n = self.K.shape[0]
            cuts = [n * i // self.threads for i in range(self.threads + 1)]
            self.blocks = [(cuts[i], cuts[i + 1], self.K[cuts[i]:cuts[i + 1]]) for i in range(self.threads)]
            self.pool = ThreadPoolExecutor(self.threads)

    def __call__(self, x):
        if self.pool is None:
            return self.K @ x
        y = np.empty(self.K.shape[0])

        def one(blk):
            a, b, B = blk
            y[a:b] = B @ x

        list(self.pool.map(one, self.blocks))
        return y

    def close(self):
        if self.pool is not None:
            self.pool.shutdown()
            self.pool = None


def cdm(K, ML, dt, nsteps, u0=None, v0=None, F=None, f_e=None, obs=None, t0=0.0, threads=None):
    """Run nsteps of Eq. cdm.  F is the spatial load vector (or None), scaled by ricker."""
    n = K.shape[0]
    Ku = RowBlockMatvec(K, threads)
    u0 = np.zeros(n) if u0 is None else np.asarray(u0, float)
    v0 = np.zeros(n) if v0 is None else np.asarray(v0, float)
    minv = 1.0 / ML

    def load(t):
        if F is None:
            return 0.0
        return F * ricker(t, f_e)

    u = u0.copy()
    u_prev = u0 - dt * v0 + 0.5 * dt * dt * minv * (load(t0) - Ku(u0))
    samples = []
    for k in range(nsteps):
        if obs is not None:
            samples.append(obs @ u)
        t = t0 + k * dt
        u_next = 2.0 * u - u_prev + dt * dt * minv * (load(t) - Ku(u))
        u_prev, u = u, u_next
    if obs is not None:
        samples.append(obs @ u)
    Ku.close()
    return u, u_prev, (np.array(samples) if obs is not None else None)


def newmark(K, M, dt, nsteps, beta=0.25, gamma=0.5, u0=None, v0=None, F=None, f_e=None,
            obs=None):
    """Algorithm 1."""
    n = K.shape[0]
    u = np.zeros(n) if u0 is None else np.asarray(u0, float).copy()
    v = np.zeros(n) if v0 is None else np.asarray(v0, float).copy()

    def load(t):
        return 0.0 if F is None else F * ricker(t, f_e)

    S = (M + beta * dt * dt * K).tocsc()
    Sfac = spla.splu(S)
    a = spla.splu(M.tocsc()).solve(load(0.0) - K @ u)
    samples = []
    for k in range(nsteps):
        if obs is not None:
            samples.append(obs @ u)
        u_pred = u + dt * v + (0.5 - beta) * dt * dt * a
        v_pred = v + (1.0 - gamma) * dt * a
        a = Sfac.solve(load((k + 1) * dt) - K @ u_pred)
        v = v_pred + gamma * dt * a
        u = u_pred + beta * dt * dt * a
    if obs is not None:
        samples.append(obs @ u)
    return u, v, a, (np.array(samples) if obs is not None else None)


class ImexSystem:
    """Partitioned operators of Sec. 2.6 for a given dt."""

    def __init__(self, K, ML_uncut_diag, Mcons, c_idx, dt, beta=0.25):
        n = K.shape[0]
        self.n = n
        self.c = np.asarray(c_idx, dtype=np.int64)
        mask = np.ones(n, dtype=bool)
        mask[self.c] = False
        self.d = np.nonzero(mask)[0]
        K = K.tocsr()
        self.Kd = K[self.d, :]
        self.Kc = K[self.c, :]
        self.Mdd = ML_uncut_diag[self.d]
        Mcc = Mcons.tocsr()[self.c, :][:, self.c]
        Kcc = K[self.c, :][:, self.c]
        self.Mcc = Mcc
        self.S = (Mcc + beta * dt * dt * Kcc).tocsc()
        self.beta = beta
        self.dt = dt


def imex(sys_, nsteps, u0=None, v0=None, F=None, f_e=None, obs=None, gamma=0.5, solver="lu"):
    """Algorithm 2 (beta = 1/4, gamma = 1/2).  ``solver`` solves S a = r by a sparse LU
    factorisation ("lu", SuperLU) or a dense Cholesky factorisation ("cholesky", LAPACK; small
    c-sets): two backward-stable solvers whose difference measures the conditioning of S."""
    n, dt, beta = sys_.n, sys_.dt, sys_.beta
    d, c = sys_.d, sys_.c
    u = np.zeros(n) if u0 is None else np.asarray(u0, float).copy()
    v = np.zeros(n) if v0 is None else np.asarray(v0, float).copy()

    def load(t):
        return np.zeros(n) if F is None else F * ricker(t, f_e)

    Sfac = None
    if len(c) and solver == "cholesky":
        import scipy.linalg as sla
        cf = sla.cho_factor(sys_.S.toarray(), lower=True)

        class _Chol:
            def solve(self, b):
                return sla.cho_solve(cf, b)

        Sfac = _Chol()
    elif len(c):
        Sfac = spla.splu(sys_.S)
    F0 = load(0.0)
    # CDM history for the d part (start-up as in cdm)
    minv_d = 1.0 / sys_.Mdd
    u_prev_d = u[d] - dt * v[d] + 0.5 * dt * dt * minv_d * (F0[d] - sys_.Kd @ u)
    vc = v[c].copy()
    ac = spla.splu(sys_.Mcc.tocsc()).solve(F0[c] - sys_.Kc @ u) if len(c) else np.zeros(0)
    samples = []
    for k in range(nsteps):
        if obs is not None:
            samples.append(obs @ u)
        Fk = load(k * dt)
        Fk1 = load((k + 1) * dt)
        # explicit step on d
        ud_next = 2.0 * u[d] - u_prev_d + dt * dt * minv_d * (Fk[d] - sys_.Kd @ u)
        u_prev_d = u[d].copy()
        # implicit step on c
        pred = u.copy()
        pred[d] = ud_next
        if len(c):
            pred_c = u[c] + dt * vc + (0.5 - beta) * dt * dt * ac
            vpred_c = vc + (1.0 - gamma) * dt * ac
            pred[c] = pred_c
            ac = Sfac.solve(Fk1[c] - sys_.Kc @ pred)
            vc = vpred_c + gamma * dt * ac
            pred[c] = pred_c + beta * dt * dt * ac
        u = pred
    if obs is not None:
        samples.append(obs @ u)
    return u, (np.array(samples) if obs is not None else None)
