"""Failure detection without a GPU fault (GPU).

* An allocation failure is injected on the host: the ``dev_alloc`` callback returns NULL at
  its k-th call.  ``ibfem_create`` and ``ibfem_upload`` must return IBFEM_ERR_OOM and give
  back every byte they had taken (the callback's live allocations fall to zero); an
  upload that failed leaves a host-only handle that uploads once memory is there.
* A bounded device wait runs out: ``ibfem_check_bounded_wait`` waits on an mbarrier that
  nothing arrives on, with a host-set poll limit; the kernel gives up, records the timeout
  and returns, ``ibfem_sync`` reports IBFEM_ERR_TIMEOUT, the context stays usable, and a new
  initial state clears the record.
* The serving loop on the GPU backend rejects a request whose device footprint exceeds its
  budget, while a request that fits completes.
"""
import numpy as np
import pytest

from helpers import SMALL_CASES
from paper_2501_19013_gb300 import workloads as W

pytestmark = pytest.mark.gpu


class FailingAllocator:
    """torch's caching allocator that fails at its k-th call (1-based; 0 = never)."""

    def __init__(self, fail_at):
        import torch
        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = set()

    def alloc(self, nbytes):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes), 0)
        self.live.add(p)
        return p

    def free(self, p):
        self.live.discard(p)
        self.torch.cuda.caching_allocator_delete(p)


def _count_allocations(w, precision):
    from paper_2501_19013_gb300 import ibfem as ib
    a = FailingAllocator(0)
    s = ib.from_workload(w, precision=precision, allocator=(a.alloc, a.free))
    n = a.calls
    s.close()
    assert not a.live
    return n


@pytest.mark.parametrize("precision", ["fp64", "exact"])
def test_create_returns_oom_and_frees_everything(precision):
    from paper_2501_19013_gb300 import ibfem as ib
    w = SMALL_CASES["elastic_evs"]()
    n = _count_allocations(w, precision)
    assert n > 3
    for k in sorted({1, 2, n // 2, n - 1, n}):
        a = FailingAllocator(k)
        with pytest.raises(ib.IbfemError) as err:
            ib.from_workload(w, precision=precision, allocator=(a.alloc, a.free))
        assert err.value.code == ib.ERR_OOM, (k, err.value)
        assert a.live == set(), f"allocation {k} of {n} failed: {len(a.live)} buffers not freed"


def test_upload_returns_oom_and_stays_host_only():
    from paper_2501_19013_gb300 import ibfem as ib
    w = SMALL_CASES["plate_one_hole"]()
    n = _count_allocations(w, "exact")
    a = FailingAllocator(n // 2)
    s = ib.from_workload(w, precision="exact", host_only=True, allocator=(a.alloc, a.free))
    with pytest.raises(ib.IbfemError) as err:
        s.upload()
    assert err.value.code == ib.ERR_OOM
    assert a.live == set()
    s.upload()                      # the failing call is past: the upload now succeeds
    s.set_dt(1e-3)
    s.set_initial()
    s.step(4)
    s.sync()
    s.close()
    assert a.live == set()


def test_bounded_wait_gives_up_and_reports_timeout():
    from paper_2501_19013_gb300 import ibfem as ib
    w = SMALL_CASES["plate_one_hole"]()
    s = ib.from_workload(w, precision="exact")
    s.set_dt(1e-3)
    s.set_initial()
    s.check_bounded_wait(1000)
    with pytest.raises(ib.IbfemError) as err:
        s.sync()
    assert err.value.code == ib.ERR_TIMEOUT
    with pytest.raises(ib.IbfemError):
        s.check_bounded_wait(0)      # the limit is checked on the host
    s.set_initial()                  # a new run clears the record; the context still works
    s.step(8)
    s.sync()
    u, _ = s.get_state()
    assert np.all(np.isfinite(u))
    s.close()


def test_serving_rejects_a_request_beyond_the_budget_on_the_gpu():
    from paper_2501_19013_gb300.serve import Request, Server, TcBackend
    small = W.plate_one_hole().with_(steps=64)
    big = W.plate_holes_elastic(n=64, p=4, count=4, steps=64)
    be = TcBackend()
    fp_small = be.setup(Request(rid=-1, arrival=0.0, workload=small, steps=64))
    be.release(fp_small[0])
    budget = int(fp_small[1] * 1.5)
    reqs = [Request(rid=0, arrival=0.0, workload=big, steps=64),
            Request(rid=1, arrival=0.0, workload=small, steps=64)]
    st = Server(be, hbm_budget=budget, max_members=4, chunk=32, workers=2).run(reqs)
    be.close()
    assert reqs[0].error == "footprint exceeds the device budget"
    assert reqs[0].footprint > budget
    assert reqs[1].error is None and reqs[1].result is not None
    assert st.summary()["completed"] == 1 and st.summary()["failed"] == 1
