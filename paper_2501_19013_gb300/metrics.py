"""Accuracy measure of the paper (Sec. 3.2, Eq. error) on observer time series.

e_{n_s} is the mean over the n_p observers of the relative L2 error of each observer's
series, taken at n_s equidistant instants t_1 .. t_{n_s} of the run.  A series here is what
``ibfem_sample`` returns: row k = Psi(t_k), k = 0 .. N, one column per observer and
component.  For several components (plane strain) an observer's series holds all of its
components (the vector norm over instants and components); observers whose reference
series is zero are left out of the mean.
"""
from __future__ import annotations

import numpy as np


def sample_rows(n_steps: int, n_s: int) -> np.ndarray:
    """Rows of the instants t_j = j T / n_s, j = 1 .. n_s, of a run of n_steps steps (the
    nearest step when n_s does not divide n_steps)."""
    if n_s < 1 or n_steps < 1:
        raise ValueError("n_s and n_steps must be >= 1")
    return np.rint(np.arange(1, n_s + 1) * (n_steps / n_s)).astype(np.int64)


def observer_error(series, ref, n_s: int, ncomp: int = 1) -> float:
    """e_{n_s} of ``series`` against ``ref`` (both (N + 1) x (n_p ncomp), Eq. error)."""
    a = np.asarray(series, dtype=np.float64)
    b = np.asarray(ref, dtype=np.float64)
    if a.shape != b.shape or a.ndim != 2 or a.shape[1] % ncomp:
        raise ValueError("series and ref must have equal (N + 1, n_p * ncomp) shapes")
    rows = sample_rows(a.shape[0] - 1, n_s)
    n_p = a.shape[1] // ncomp
    errs = []
    for i in range(n_p):
        cols = slice(i * ncomp, (i + 1) * ncomp)
        r = b[rows, cols]
        nr = np.linalg.norm(r)
        if nr > 0:
            errs.append(np.linalg.norm(a[rows, cols] - r) / nr)
    return float(np.mean(errs)) if errs else 0.0
