"""Accuracy measure of the paper (Sec. 3.2, Eq. error) on observer time series.

e_{n_s} is the mean over the n_p observers of the relative L2 error of each observer's
series, taken at n_s equidistant instants t_1 .. t_{n_s} of the run.  A series here is what
``ibfem_sample`` returns: row k = Psi(t_k), k = 0 .. N, one column per observer and
component.  For several components (plane strain) an observer's series holds all of its
components (the vector norm over instants and components).

Observers that the wave has not reached by the end of the run hold only the exponentially
small precursor of the pulse; their relative error is noise and says nothing about the
arithmetic.  So an observer whose reference norm lies below ``floor`` times the largest
observer norm of the run is left out of the mean (``floor = 1e-8`` by default; a zero
reference series is always left out), and ``observer_errors`` reports how many were.
"""
from __future__ import annotations

import numpy as np


def sample_rows(n_steps: int, n_s: int) -> np.ndarray:
    """Rows of the instants t_j = j T / n_s, j = 1 .. n_s, of a run of n_steps steps (the
    nearest step when n_s does not divide n_steps)."""
    if n_s < 1 or n_steps < 1:
        raise ValueError("n_s and n_steps must be >= 1")
    return np.rint(np.arange(1, n_s + 1) * (n_steps / n_s)).astype(np.int64)


def observer_errors(series, ref, n_s: int, ncomp: int = 1, floor: float = 1e-8) -> dict:
    """Per-observer relative L2 errors of ``series`` against ``ref`` at the n_s instants
    (both (N + 1) x (n_p ncomp)); ``mean`` is e_{n_s} over the observers kept (reference
    norm above ``floor`` times the largest), ``per_observer`` holds None for the others."""
    a = np.asarray(series, dtype=np.float64)
    b = np.asarray(ref, dtype=np.float64)
    if a.shape != b.shape or a.ndim != 2 or a.shape[1] % ncomp:
        raise ValueError("series and ref must have equal (N + 1, n_p * ncomp) shapes")
    rows = sample_rows(a.shape[0] - 1, n_s)
    n_p = a.shape[1] // ncomp
    norms = [float(np.linalg.norm(b[rows, i * ncomp:(i + 1) * ncomp])) for i in range(n_p)]
    big = max(norms) if norms else 0.0
    per = []
    for i in range(n_p):
        cols = slice(i * ncomp, (i + 1) * ncomp)
        if norms[i] > 0.0 and norms[i] > floor * big:
            per.append(float(np.linalg.norm(a[rows, cols] - b[rows, cols]) / norms[i]))
        else:
            per.append(None)
    kept = [e for e in per if e is not None]
    return {"mean": float(np.mean(kept)) if kept else 0.0, "per_observer": per,
            "left_out": n_p - len(kept), "floor": floor}


def observer_error(series, ref, n_s: int, ncomp: int = 1, floor: float = 1e-8) -> float:
    """e_{n_s} of ``series`` against ``ref`` (both (N + 1) x (n_p ncomp), Eq. error), over
    the observers whose reference norm exceeds ``floor`` times the largest."""
    return observer_errors(series, ref, n_s, ncomp, floor)["mean"]
