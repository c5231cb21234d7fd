"""The paper's observer error e_{n_s} (Sec. 3.2, Eq. error) on hand-made series."""
import numpy as np
import pytest

from paper_2501_19013_gb300.metrics import observer_error, observer_errors, sample_rows


def test_sample_rows_are_the_equidistant_instants():
    assert list(sample_rows(10000, 100)[:3]) == [100, 200, 300]
    assert sample_rows(10000, 100)[-1] == 10000
    assert list(sample_rows(6, 6)) == [1, 2, 3, 4, 5, 6]       # n_s = N: every step but t_0


def test_observer_error_closed_forms():
    t = np.linspace(0.0, 1.0, 1001)
    ref = np.stack([np.sin(7 * t), np.cos(3 * t), 2 + t], axis=1)
    # a uniform relative perturbation c of every series gives e = |c|
    assert observer_error(1.03 * ref, ref, 100) == pytest.approx(0.03, rel=1e-12)
    # per-observer factors average: (0.01 + 0.02 + 0.06) / 3
    f = np.array([1.01, 0.98, 1.06])
    assert observer_error(ref * f, ref, 1000) == pytest.approx(0.03, rel=1e-12)
    # only the sampled instants count: a change at t_0 alone is invisible
    a = ref.copy()
    a[0] += 5.0
    assert observer_error(a, ref, 100) == 0.0
    # a change off the n_s = 100 grid is invisible to e_100 and seen by e_1000
    a = ref.copy()
    a[5, 0] += 1.0
    assert observer_error(a, ref, 100) == 0.0
    assert observer_error(a, ref, 1000) > 0.0


def test_observer_error_components_and_zero_reference():
    t = np.linspace(0.0, 1.0, 101)
    ref = np.stack([np.sin(5 * t), np.cos(5 * t), np.zeros_like(t), np.zeros_like(t)], axis=1)
    a = ref.copy()
    a[:, 1] *= 1.1
    # observer 0 holds columns 0 and 1; observer 1 (zero reference) is left out
    r = sample_rows(100, 100)
    want = np.linalg.norm(a[r, :2] - ref[r, :2]) / np.linalg.norm(ref[r, :2])
    assert observer_error(a, ref, 100, ncomp=2) == pytest.approx(want, rel=1e-12)
    with pytest.raises(ValueError):
        observer_error(a[:, :3], ref[:, :3], 100, ncomp=2)


def test_observers_the_wave_has_not_reached_are_left_out():
    """An observer whose reference series is 1e-12 of the others' (the precursor of a pulse
    that has not arrived) is left out of the mean, and counted; at floor 0 it is kept and
    its relative error (noise) dominates."""
    t = np.linspace(0.0, 1.0, 201)
    ref = np.stack([np.sin(9 * t), np.cos(4 * t), 1e-12 * np.sin(3 * t)], axis=1)
    a = ref * np.array([1.0 + 1e-6, 1.0 - 2e-6, 1.0])
    a[:, 2] += 1e-12            # relative noise of 1 on the unreached observer
    r = observer_errors(a, ref, 100)
    assert r["left_out"] == 1 and r["per_observer"][2] is None
    assert r["mean"] == pytest.approx(1.5e-6, rel=1e-6)
    assert observer_error(a, ref, 100) == r["mean"]
    assert observer_error(a, ref, 100, floor=0.0) > 0.1
