"""Continuous-batching request loop over the batched tensor-core path.

Requests (a workload plus a step count) arrive over time.  Each one goes through

    arrival -> host setup (worker thread: discretisation on the host, footprint known)
            -> admission (main loop, FIFO: a free slot and enough device memory left
               in the budget; the footprint is reserved)
            -> device init (worker thread: upload, critical time step, source,
               observers, initial state)
            -> join the batch (main loop, between chunks of batched steps)
            -> finish (its step budget used up; it leaves the batch)
            -> read-back (worker thread: the observer series to the host) and release
               (device memory back to the budget).

Latency is read-back time minus arrival time.  The loop never waits for a request: it
keeps enqueueing chunks of batched steps while members are active, with back-pressure
(at most ``max_pending`` chunks on the GPU), and admits new work between chunks, so
requests that arrive while others run join them on the device.

The scheduler is written against a small backend interface so that its logic can be
tested without a GPU; ``TcBackend`` is the GPU implementation (ibfem_upload /
ibfem_batch_*).
"""
from __future__ import annotations

import math
import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Any, Callable, List, Optional

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the run
    workload: Any
    steps: int
    # filled in by the server (seconds after the start of the run)
    t_setup: float = math.nan      # host setup done
    t_admit: float = math.nan      # admitted (memory reserved)
    t_join: float = math.nan       # joined the batch
    t_finish: float = math.nan     # left the batch (all steps enqueued)
    t_done: float = math.nan       # result on the host
    footprint: int = 0
    n_dof: int = 0
    dt: float = math.nan
    tile_variant: int = 0
    error: Optional[str] = None
    result: Any = None

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


class Backend:
    """What the scheduler needs from the solver side (all handles are opaque)."""

    def setup(self, req: Request):                 # worker: -> (handle, footprint bytes, n_dof)
        raise NotImplementedError

    def init(self, req: Request, handle) -> None:  # worker: device buffers, dt, source, initial state
        raise NotImplementedError

    def join(self, req: Request, handle) -> None:  # main loop
        raise NotImplementedError

    def run(self, n: int) -> None:                 # main loop: enqueue n batched steps
        raise NotImplementedError

    def poll(self) -> list:                        # main loop: handles that left the batch
        raise NotImplementedError

    def wait(self, max_pending: int) -> None:      # main loop: back-pressure
        raise NotImplementedError

    def collect(self, req: Request, handle):      # worker: read the result back (blocks)
        raise NotImplementedError

    def release(self, handle) -> None:             # worker: free the device memory
        raise NotImplementedError

    def close(self) -> None:
        pass


@dataclass
class ServeStats:
    requests: List[Request] = field(default_factory=list)
    wall_s: float = 0.0
    chunks: int = 0
    max_members: int = 0

    def summary(self) -> dict:
        ok = [r for r in self.requests if r.error is None and not math.isnan(r.t_done)]
        lat = np.array([r.latency for r in ok]) if ok else np.zeros(0)
        work = float(sum(r.n_dof * r.steps for r in ok))
        span = (max(r.t_done for r in ok) - min(r.arrival for r in ok)) if ok else 0.0
        q = lambda a, f: float(np.percentile(a, f)) if len(a) else None
        stage = lambda f: q(np.array([f(r) for r in ok]), 50) if ok else None
        return {
            "requests": len(self.requests), "completed": len(ok),
            "failed": sum(r.error is not None for r in self.requests),
            "p50_s": q(lat, 50), "p99_s": q(lat, 99), "max_s": float(lat.max()) if len(lat) else None,
            "dof_steps_per_s": work / span if span > 0 else None,
            "span_s": span, "wall_s": self.wall_s, "chunks": self.chunks,
            "max_concurrent": self.max_members,
            "p50_stage_s": {"setup": stage(lambda r: r.t_setup - r.arrival),
                            "admit_wait": stage(lambda r: r.t_admit - r.t_setup),
                            "init": stage(lambda r: r.t_join - r.t_admit),
                            "in_batch": stage(lambda r: r.t_finish - r.t_join),
                            "readback": stage(lambda r: r.t_done - r.t_finish)},
        }


class Server:
    """FIFO admission by device-memory footprint into a continuous batch."""

    def __init__(self, backend: Backend, hbm_budget: int, max_members: int = 64,
                 chunk: int = 32, max_pending: int = 2, workers: int = 8,
                 clock: Callable[[], float] = time.perf_counter, idle_sleep: float = 5e-4):
        self.be = backend
        self.budget = int(hbm_budget)
        self.max_members = int(max_members)
        self.chunk = int(chunk)
        self.max_pending = int(max_pending)
        self.workers = int(workers)
        self.clock = clock
        self.idle_sleep = idle_sleep

    def run(self, requests: List[Request]) -> ServeStats:
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        stats = ServeStats(requests=reqs)
        pool = ThreadPoolExecutor(max_workers=self.workers)
        t0 = self.clock()
        now = lambda: self.clock() - t0
        nxt = 0                      # next request to arrive
        setting_up = deque()         # (req, future) in arrival order
        ready = deque()              # (req, handle): footprint known, waiting for admission
        initing = deque()            # (req, handle, future)
        collecting = []              # (req, handle, future)
        handle_req = {}              # id(handle) -> (req, handle)
        used = 0                     # reserved device bytes
        admitted = 0                 # admitted and not yet released
        in_batch = 0
        done = 0
        try:
            while done < len(reqs):
                t = now()
                # arrivals -> host setup
                while nxt < len(reqs) and reqs[nxt].arrival <= t:
                    r = reqs[nxt]
                    setting_up.append((r, pool.submit(self.be.setup, r)))
                    nxt += 1
                # host setups that finished (kept in arrival order)
                while setting_up and setting_up[0][1].done():
                    r, f = setting_up.popleft()
                    try:
                        h, fp, nd = f.result()
                    except Exception as e:   # a request that cannot be set up fails alone
                        r.error, r.t_done = f"setup: {e}", now()
                        done += 1
                        continue
                    r.t_setup, r.footprint, r.n_dof = now(), int(fp), int(nd)
                    if r.footprint > self.budget:
                        r.error, r.t_done = "footprint exceeds the device budget", now()
                        pool.submit(self.be.release, h)
                        done += 1
                        continue
                    ready.append((r, h))
                # admission (FIFO: the head waits until it fits)
                while ready and admitted < self.max_members and used + ready[0][0].footprint <= self.budget:
                    r, h = ready.popleft()
                    used += r.footprint
                    admitted += 1
                    r.t_admit = now()
                    initing.append((r, h, pool.submit(self.be.init, r, h)))
                # device inits that finished -> join the batch
                still = deque()
                for r, h, f in initing:
                    if not f.done():
                        still.append((r, h, f))
                        continue
                    try:
                        f.result()
                        self.be.join(r, h)
                        r.t_join = now()
                        handle_req[id(h)] = (r, h)
                        in_batch += 1
                    except Exception as e:
                        r.error = f"init: {e}"
                        collecting.append((r, h, pool.submit(self.be.release, h)))
                initing = still
                stats.max_members = max(stats.max_members, in_batch)
                # one chunk of batched steps, with back-pressure
                if in_batch > 0:
                    self.be.run(self.chunk)
                    stats.chunks += 1
                    for h in self.be.poll():
                        r, _ = handle_req.pop(id(h))
                        r.t_finish = now()
                        in_batch -= 1
                        collecting.append((r, h, pool.submit(self._collect_release, r, h)))
                    self.be.wait(self.max_pending)
                # read-backs that finished -> memory back to the budget
                keep = []
                for r, h, f in collecting:
                    if not f.done():
                        keep.append((r, h, f))
                        continue
                    try:
                        f.result()
                    except Exception as e:
                        if r.error is None:
                            r.error = f"collect: {e}"
                    r.t_done = now()
                    used -= r.footprint
                    admitted -= 1
                    done += 1
                collecting = keep
                if in_batch == 0:
                    time.sleep(self.idle_sleep)
        finally:
            pool.shutdown(wait=True)
        stats.wall_s = now()
        return stats

    def _collect_release(self, r: Request, h):
        try:
            r.result = self.be.collect(r, h)
        finally:
            self.be.release(h)


class TcBackend(Backend):
    """GPU backend: exact tensor-core solvers in one ``ibfem`` batch."""

    def __init__(self, device: int = 0, dt_factor: float = 0.9, keep_state: bool = False,
                 dt_fn: Optional[Callable[[Any], float]] = None, autotune: bool = True):
        import threading
        from . import ibfem
        self.ib = ibfem
        self.batch = ibfem.Batch(device=device)
        self.device = device
        self.dt_factor = dt_factor
        self.keep_state = keep_state
        self.dt_fn = dt_fn
        self.autotune = autotune
        self.tiles = {}                  # (dim, cells, p, physics) -> tile variant
        self.tiles_lock = threading.Lock()

    def setup(self, r: Request):
        w = r.workload
        s = self.ib.from_workload(w, precision="exact", host_only=True, device=self.device)
        inf = s.info()
        nobs = 0 if w.observers is None else len(w.observers)
        ring = (r.steps + 1) * max(nobs * inf.ncomp, 1) * 8
        return s, int(inf.device_bytes) + ring + (1 << 16), int(inf.n_dof)

    def init(self, r: Request, s) -> None:
        w = r.workload
        s.upload()
        if self.autotune:
            # tile shape by the autotuner, once per problem shape (later ones reuse it)
            key = (w.dim, tuple(w.n), w.p, w.physics)
            with self.tiles_lock:
                v = self.tiles.get(key)
            if v is None:
                v, _ = s.autotune(reps=3)
                with self.tiles_lock:
                    self.tiles[key] = v
            else:
                s.set_tile_variant(v)
            r.tile_variant = v
        if self.dt_fn is not None:
            dt = self.dt_fn(s)
        else:
            dt_crit, _, _ = s.crit_dt(max_iter=400, rtol=1e-8)
            dt = self.dt_factor * dt_crit
        s.set_dt(dt)
        kind, params = self.ib.source_params(w)
        s.set_source(kind, params, w.f0)
        if w.observers is not None and len(w.observers):
            s.set_observers(w.observers, r.steps + 1)
        s.set_initial()
        r.dt = dt

    def join(self, r: Request, s) -> None:
        self.batch.add(s, r.steps)

    def run(self, n: int) -> None:
        self.batch.run(n)

    def poll(self) -> list:
        return self.batch.poll()

    def wait(self, max_pending: int) -> None:
        self.batch.wait(max_pending)

    def collect(self, r: Request, s):
        series = s.sample(r.steps + 1) if getattr(s, "n_obs", 0) else None
        s.sync()   # raises on a diverged state
        if self.keep_state:
            return series, s.get_state()[0]
        return series

    def release(self, s) -> None:
        s.close()

    def close(self) -> None:
        self.batch.close()
