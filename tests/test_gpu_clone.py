"""Several loads on one discretisation: ``ibfem_clone`` (GPU).

A clone shares the device geometry and matrices of its source and owns its state, load,
observers and dt^2 / M_L.  Its arithmetic is that of a handle built from scratch on the
same inputs, so its results must equal such a handle's bit for bit, whether it steps
alone, after its source was destroyed, or in a batch next to its source and its siblings.
One clone with a load of its own is also checked against the oracle's CDM (Eq. cdm).
"""
import numpy as np
import pytest

from helpers import gpu_solver, oracle_cdm, oracle_disc, oracle_dt, rel_l2
from paper_2501_19013_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _cases():
    return [
        W.plate_holes_elastic(n=24, p=4, count=3, steps=120),     # 2D elastic, edge traction
        W.porous_voxel(n=7, vn=14, p=2, seed=2, steps=70),        # 3D voxels, point source
        W.plate_one_hole().with_(steps=100),                      # 2D scalar
    ]


def _loads(w, k):
    """k point loads at distinct kept positions (the workload's observer points)."""
    return [{"kind": "point", "x": list(map(float, w.observers[i % len(w.observers)]))}
            for i in range(k)]


def _set_load(s, w, load):
    from paper_2501_19013_gb300 import ibfem as ib
    kind, params = ib.source_params(w.with_(source=load))
    s.set_source(kind, params, w.f0)


def _fresh(w, precision, dt, load, steps, variant=0):
    s = gpu_solver(w.with_(source=load), precision)
    s.set_observers(w.observers, steps + 1)
    s.set_dt(dt)
    if precision != "fp64":
        s.set_tile_variant(variant)
    s.set_initial()
    s.step(steps)
    s.sync()
    u, up = s.get_state()
    ser = s.sample(steps + 1)
    s.close()
    return u, up, ser


@pytest.mark.parametrize("precision", ["fp64", "exact"])
def test_clone_equals_fresh_handle_after_source_is_gone(precision):
    for w in _cases():
        src = gpu_solver(w, precision)
        dt = 0.9 * src.crit_dt(max_iter=300, rtol=1e-8)[0]
        src.set_dt(dt)
        c = src.clone()
        inf_s, inf_c = src.info(), c.info()
        assert inf_c.shared_device_bytes == inf_s.shared_device_bytes > 0, w.name
        assert inf_c.dt == dt and inf_c.n_dof == inf_s.n_dof
        # the clone's own arrays are the per-load part only
        assert inf_c.device_bytes - inf_c.shared_device_bytes < inf_s.device_bytes - inf_s.shared_device_bytes
        src.close()                                   # the shared arrays stay alive
        load = _loads(w, 2)[1]
        _set_load(c, w, load)
        c.set_observers(w.observers, w.steps + 1)
        c.set_initial()
        c.step(w.steps)
        c.sync()
        u, up = c.get_state()
        ser = c.sample(w.steps + 1)
        c.close()
        uf, upf, serf = _fresh(w, precision, dt, load, w.steps)
        assert np.array_equal(u, uf), (w.name, precision)
        assert np.array_equal(up, upf), (w.name, precision)
        assert np.array_equal(ser, serf), (w.name, precision)
        assert np.abs(u).max() > 0


def test_clone_with_its_own_load_matches_the_oracle():
    w = W.plate_one_hole().with_(steps=150)
    load = _loads(w, 3)[2]
    d = oracle_disc(w)
    dt = oracle_dt(d)
    u_o, _, s_o = oracle_cdm(w.with_(source=load), d, dt, w.steps)
    src = gpu_solver(w, "fp64")
    src.set_dt(dt)
    c = src.clone()
    _set_load(c, w, load)
    c.set_observers(w.observers, w.steps + 1)
    c.set_initial()
    # the source keeps its own load and state: step both, interleaved on their streams
    src.set_initial()
    src.step(w.steps)
    c.step(w.steps)
    c.sync()
    u_c, _ = c.get_state()
    s_c = c.sample(w.steps + 1)
    src.sync()
    u_s, _ = src.get_state()
    assert rel_l2(u_c, u_o) <= 1e-10
    assert rel_l2(s_c, s_o) <= 1e-10
    u_so, _, _ = oracle_cdm(w, d, dt, w.steps)
    assert rel_l2(u_s, u_so) <= 1e-10
    c.close()
    src.close()


def test_clones_in_one_batch_equal_fresh_handles():
    """A source and its clones, each with another load, as members of one batched launch:
    each equals its fresh single-problem run bitwise; a clone of a tile-variant-1 source
    keeps that tile shape."""
    from paper_2501_19013_gb300 import ibfem as ib
    for w, variant in zip(_cases()[:2], (0, 1)):
        src = gpu_solver(w, "exact")
        src.set_tile_variant(variant)
        dt = 0.9 * src.crit_dt(max_iter=300, rtol=1e-8)[0]
        src.set_dt(dt)
        loads = _loads(w, 4)
        members = [src] + [src.clone() for _ in loads[1:]]
        steps = [w.steps - 10 * k for k in range(len(members))]
        for s, load in zip(members, loads):
            assert s.info().tile_variant == variant
            _set_load(s, w, load)
            s.set_observers(w.observers, w.steps + 1)
            s.set_initial()
        b = ib.Batch()
        for s, n in zip(members, steps):
            b.add(s, n)
        done = []
        for _ in range(40):
            b.run(32)
            done += b.poll()
            if len(done) == len(members):
                break
        assert len(done) == len(members)
        assert b.status()[0] == 0
        b.close()
        for s, load, n in zip(members, loads, steps):
            s.sync()
            u, up = s.get_state()
            ser = s.sample(n + 1)
            uf, upf, serf = _fresh(w, "exact", dt, load, n, variant)
            assert np.array_equal(u, uf), (w.name, n)
            assert np.array_equal(up, upf), (w.name, n)
            assert np.array_equal(ser, serf), (w.name, n)
        for s in members:
            s.close()


def test_clone_refuses_a_c_set_handle():
    from paper_2501_19013_gb300 import ibfem as ib
    w = W.plate_holes_imex(n=30, p=3, count=3, scheme="imex", steps=10)
    s = ib.from_workload(w)
    assert s.info().n_c > 0
    with pytest.raises(ib.IbfemError) as ei:
        s.clone()
    assert ei.value.code == ib.ERR_ARG
    s.close()
