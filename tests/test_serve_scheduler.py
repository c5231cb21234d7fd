"""Host logic of the continuous-batching request loop, against a fake backend (no GPU).

The fake mirrors the batch semantics of the C library: ``run(n)`` advances every member by
up to n steps, a member whose budget is used up leaves the batch and is returned by
``poll``.  The tests check FIFO admission by device-memory footprint, the member limit,
exact step budgets, continuous admission (requests joining while others run) and that a
request larger than the budget fails alone.
"""
import threading
import time

import pytest

from paper_2501_19013_gb300.serve import Backend, Request, Server


class FakeBackend(Backend):
    def __init__(self, footprints, n_dof=1000):
        self.fp = footprints
        self.n_dof = n_dof
        self.lock = threading.Lock()
        self.live = 0            # bytes of initialised, not yet released handles
        self.max_live = 0
        self.members = {}        # handle -> remaining steps
        self.finished = []
        self.steps_done = {}
        self.max_members = 0
        self.join_order = []
        self.handles = {}

    def setup(self, r):
        time.sleep(0.001)
        return {"rid": r.rid}, self.fp[r.rid], self.n_dof

    def init(self, r, h):
        with self.lock:
            h["live"] = True
            self.live += r.footprint
            self.max_live = max(self.max_live, self.live)
        time.sleep(0.001)

    def join(self, r, h):
        self.members[h["rid"]] = r.steps
        self.handles[h["rid"]] = h
        self.steps_done[h["rid"]] = 0
        self.join_order.append(h["rid"])
        self.max_members = max(self.max_members, len(self.members))

    def run(self, n):
        for rid in list(self.members):
            k = min(n, self.members[rid])
            self.members[rid] -= k
            self.steps_done[rid] += k
            if self.members[rid] == 0:
                del self.members[rid]
                self.finished.append(self.handles[rid])
        time.sleep(0.0002)

    def poll(self):
        out, self.finished = self.finished, []
        return out

    def wait(self, max_pending):
        pass

    def collect(self, r, h):
        return r.rid

    def release(self, h):
        with self.lock:
            if h.get("live"):
                self.live -= self.fp[h["rid"]]


def _requests(n, gap=0.002, steps=(100, 400)):
    return [Request(rid=i, arrival=i * gap, workload=None, steps=steps[0] + (37 * i) % (steps[1] - steps[0]))
            for i in range(n)]


def test_all_requests_complete_with_exact_step_budgets():
    reqs = _requests(20)
    be = FakeBackend({r.rid: 10 for r in reqs})
    st = Server(be, hbm_budget=1000, max_members=8, chunk=32).run(reqs)
    assert all(r.error is None for r in st.requests)
    for r in st.requests:
        assert be.steps_done[r.rid] == r.steps
        assert r.arrival <= r.t_setup <= r.t_admit <= r.t_join <= r.t_finish <= r.t_done
        assert r.result == r.rid
    s = st.summary()
    assert s["completed"] == 20 and s["p50_s"] <= s["p99_s"]


def test_footprint_budget_and_member_limit_hold():
    reqs = _requests(24)
    fp = {r.rid: 100 + 50 * (r.rid % 4) for r in reqs}
    be = FakeBackend(fp)
    budget = 450
    st = Server(be, hbm_budget=budget, max_members=3, chunk=16).run(reqs)
    assert all(r.error is None for r in st.requests)
    assert be.max_live <= budget
    assert be.max_members <= 3


def test_admission_is_fifo():
    reqs = _requests(16)
    be = FakeBackend({r.rid: 100 for r in reqs})
    st = Server(be, hbm_budget=250, max_members=64, chunk=32).run(reqs)
    by_admit = sorted(st.requests, key=lambda r: r.t_admit)
    assert [r.rid for r in by_admit] == sorted(r.rid for r in st.requests)


def test_requests_join_while_others_run():
    reqs = _requests(12, gap=0.003, steps=(2000, 3000))
    be = FakeBackend({r.rid: 1 for r in reqs})
    st = Server(be, hbm_budget=100, max_members=64, chunk=32).run(reqs)
    overlaps = 0
    rs = st.requests
    for a in rs:
        for b in rs:
            if a.rid != b.rid and a.t_join < b.t_join < a.t_finish:
                overlaps += 1
    assert overlaps > 0
    assert st.max_members > 1


def test_oversized_request_fails_alone():
    reqs = _requests(6)
    fp = {r.rid: 10 for r in reqs}
    fp[2] = 10 ** 9
    be = FakeBackend(fp)
    st = Server(be, hbm_budget=1000, max_members=8, chunk=32).run(reqs)
    errs = {r.rid: r.error for r in st.requests}
    assert errs[2] is not None and "budget" in errs[2]
    assert all(errs[i] is None for i in errs if i != 2)
    assert be.live == 0


def test_setup_failure_fails_alone():
    class Failing(FakeBackend):
        def setup(self, r):
            if r.rid == 1:
                raise ValueError("bad geometry")
            return super().setup(r)

    reqs = _requests(5)
    be = Failing({r.rid: 10 for r in reqs})
    st = Server(be, hbm_budget=1000).run(reqs)
    assert st.requests[1].error.startswith("setup")
    assert sum(r.error is None for r in st.requests) == 4


def test_serving_stream_generator_is_seeded():
    from paper_2501_19013_gb300 import workloads as W
    a = W.serving_request(3)
    b = W.serving_request(3)
    assert a.name == b.name and a.steps == b.steps
    assert 500 <= a.steps <= 5000
    t = W.poisson_arrivals(200, 10.0, 0)
    assert (t[1:] > t[:-1]).all()
    assert 15.0 < t[-1] < 25.0          # mean gap 0.1 s
