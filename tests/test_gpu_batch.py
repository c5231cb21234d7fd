"""Batched stepping and the serving loop on the GPU.

A batched launch runs, per tile, the arithmetic of the single-problem exact tensor-core
kernel, so every member must end bitwise equal to the same problem stepped alone through
``ibfem_step`` -- whatever else is in the batch, whenever it joined and however the
launches were chunked.  The tolerance is therefore zero.
"""
import numpy as np
import pytest

from helpers import gpu_solver
from paper_2501_19013_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _cases():
    return [
        W.plate_holes_elastic(n=24, p=4, count=3, steps=120),                    # (2, 4, 2)
        W.plate_holes_elastic(n=19, p=2, count=2, seed=3, steps=90),             # (2, 2, 2) ragged
        W.plate_holes_imex(n=30, p=3, count=3, scheme="cdm", steps=150),         # (2, 3, 1)
        W.plate_one_hole().with_(steps=100),                                     # (2, 2, 1)
        W.plate_holes_imex(n=40, p=2, count=4, seed=5, scheme="cdm", steps=130),  # (2, 2, 1), other grid
        W.porous_voxel(n=7, vn=14, p=2, seed=2, steps=70),                       # (3, 2, 1)
        W.porous_voxel(n=9, vn=18, p=2, seed=4, steps=85),                       # (3, 2, 1), other K_ref
        W.porous_voxel(n=6, vn=12, p=3, steps=60),                               # (3, 3, 1)
    ]


def _prepared(w, dt=None, capacity=None):
    s = gpu_solver(w, "exact")
    if w.observers is not None:
        s.set_observers(w.observers, capacity or w.steps + 1)
    if dt is None:
        dt = 0.9 * s.crit_dt(max_iter=300, rtol=1e-8)[0]
    s.set_dt(dt)
    s.set_initial()
    return s, dt


def _alone(w, dt, steps, variant=0):
    s, _ = _prepared(w, dt, steps + 1)
    s.set_tile_variant(variant)
    s.step(steps)
    s.sync()
    u, up = s.get_state()
    ser = s.sample(steps + 1) if w.observers is not None else None
    s.close()
    return u, up, ser


def test_batch_members_equal_alone_bitwise():
    from paper_2501_19013_gb300 import ibfem as ib
    cases = _cases()
    members = [_prepared(w) for w in cases]
    b = ib.Batch()
    half = len(cases) // 2
    for (s, _), w in zip(members[:half], cases[:half]):
        b.add(s, w.steps)
    b.run(40)                                  # the rest joins while the first half runs
    for (s, _), w in zip(members[half:], cases[half:]):
        b.add(s, w.steps)
    done = []
    for _ in range(100):
        b.run(32)
        done += b.poll()
        if len(done) == len(cases):
            break
    assert len(done) == len(cases)
    assert b.status()[0] == 0
    for (s, dt), w in zip(members, cases):
        assert s.info().step == w.steps
        s.sync()
        u, up = s.get_state()
        ser = s.sample(w.steps + 1) if w.observers is not None else None
        ua, upa, sera = _alone(w, dt, w.steps)
        assert np.array_equal(u, ua), w.name
        assert np.array_equal(up, upa), w.name
        if ser is not None:
            assert np.array_equal(ser, sera), w.name
        assert np.abs(u).max() > 0, w.name
        s.close()
    b.close()


def test_member_calls_are_refused_and_destroy_leaves_the_batch():
    from paper_2501_19013_gb300 import ibfem as ib
    cases = _cases()[:3]
    members = [_prepared(w) for w in cases]
    b = ib.Batch()
    for (s, _), w in zip(members, cases):
        b.add(s, w.steps)
    b.run(16)
    with pytest.raises(ib.IbfemError) as ei:
        members[0][0].step(1)
    assert ei.value.code == ib.ERR_STATE
    members[1][0].close()                     # destroyed while a member
    done = []
    for _ in range(50):
        b.run(32)
        done += b.poll()
        if b.status()[0] == 0:
            break
    assert {id(s) for s in done} == {id(members[0][0]), id(members[2][0])}
    for k in (0, 2):
        s, dt = members[k]
        w = cases[k]
        s.sync()
        ua, _, _ = _alone(w, dt, w.steps)
        assert np.array_equal(s.get_state()[0], ua)
        s.close()
    b.close()


def test_upload_allocates_the_announced_footprint():
    from paper_2501_19013_gb300 import ibfem as ib
    for w in _cases()[:4] + _cases()[5:6]:
        h = ib.from_workload(w, precision="exact", host_only=True)
        planned = h.info().device_bytes
        h.upload()
        assert h.info().device_bytes == planned, w.name
        d = ib.from_workload(w, precision="exact")
        assert d.info().device_bytes == planned, w.name
        d.close()
        # an uploaded handle steps like one created on the device
        h.set_dt(1e-4)
        h.set_initial()
        h.step(3)
        h.sync()
        h.close()


def test_server_results_equal_alone():
    from paper_2501_19013_gb300.serve import Request, Server, TcBackend
    cases = _cases()[:6]
    reqs = [Request(rid=i, arrival=0.02 * i, workload=w, steps=w.steps + 7 * i)
            for i, w in enumerate(cases)]
    be = TcBackend(keep_state=True)
    st = Server(be, hbm_budget=1 << 34, max_members=4, chunk=32, workers=4).run(reqs)
    be.close()
    summ = st.summary()
    assert summ["completed"] == len(cases), [r.error for r in st.requests]
    assert summ["p50_s"] > 0 and summ["p99_s"] >= summ["p50_s"]
    for r in st.requests:
        ser, u = r.result
        ua, _, sera = _alone(r.workload, r.dt, r.steps, r.tile_variant)
        assert np.array_equal(u, ua), r.workload.name
        if ser is not None:
            assert np.array_equal(ser, sera), r.workload.name


def test_batch_mixes_tile_variants_and_equals_alone():
    """Members of one shape class with different tile shapes run as separate launches of the
    batch; each equals its own single-problem run bitwise."""
    from paper_2501_19013_gb300 import ibfem as ib
    cases = [_cases()[0], _cases()[0].with_(steps=90), _cases()[5]]
    variants = [0, 1, 1]
    members = []
    for w, v in zip(cases, variants):
        s, dt = _prepared(w)
        s.set_tile_variant(v)
        members.append((s, dt))
    b = ib.Batch()
    for (s, _), w in zip(members, cases):
        b.add(s, w.steps)
    done = []
    for _ in range(60):
        b.run(32)
        done += b.poll()
        if len(done) == len(cases):
            break
    assert len(done) == len(cases)
    for (s, dt), w, v in zip(members, cases, variants):
        s.sync()
        u, _ = s.get_state()
        a, _ = _prepared(w, dt, w.steps + 1)
        a.set_tile_variant(v)
        a.step(w.steps)
        a.sync()
        ua, _ = a.get_state()
        a.close()
        assert np.array_equal(u, ua), (w.name, v)
        s.close()
    b.close()
