"""Benchmark of the explicit immersed-boundary wave step on one or more GB300s.

Workload (the metric's configuration): 2D plane-strain elastodynamics on the unit plate
with 12 seeded holes (r in [0.02, 0.08]), 256x256 cells, p = 4 GLL elements, eigenvalue
stabilisation of cut cells (f_lambda = 1e-2, eps = 1e-4, alpha = 1e-12), Ricker edge
traction, dt = 0.9 dt_crit.  One "step" is one central-difference time step (Eq. cdm):
cut-cell mat-vec + fused element operator / assembly / update.

Metric: DOF-steps/s (kept DOFs x steps / device time).  Every timed step is preceded by an
untimed L2 eviction: a 256 MiB device write followed by a 256 MiB read of another buffer
(so that the cache holds clean lines of unrelated data; the state of this workload, ~60 MB,
would otherwise stay L2-resident).  Also reported: per-variant error against the FP64 path
after the configured 10k steps and time to that accuracy, the dominant kernel's roofline,
an end-to-end number through the C ABI with host buffers, the oracle timed on the host
cores, and SM clocks sampled during the timed region.

``--impl reference`` times the FP64 CPU oracle (the paper's assembled-matrix CDM loop) on
the same plate (set-up untimed, as in the paper's timings), on all host cores.  With
torchrun (N > 1) every rank runs its own replica of the workload (the path is replicated,
not sharded); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DOF-steps/s & time to L2 err 1e-4 (mixed vs FP64 plain, 1 GB300); p50/p99 latency"
UNIT = "DOF-steps/s"
FP64_PEAK_GFLOPS = 1250.0   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal table figure)
FLUSH_BYTES = 512 << 20    # two halves of 256 MiB, each twice the L2 cache


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ibfem_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


GRID = 256
WORKLOAD = "plate_holes_elastic"


def workload_for_bench():
    from paper_2501_19013_gb300 import workloads as W
    if WORKLOAD == "plate_holes_imex":
        return W.plate_holes_imex(n=GRID if GRID != 256 else 512)
    if WORKLOAD == "porous_voxel":
        return W.porous_voxel(n=GRID if GRID != 256 else 64)
    if WORKLOAD == "plate_one_hole":
        return W.plate_one_hole()
    if WORKLOAD == "rotated_cube":
        return W.rotated_cube(ne=GRID if GRID != 256 else 13)
    return W.plate_holes_elastic(n=GRID)


_ORACLE = {}


def oracle_disc():
    """The oracle's discretisation of the bench workload (built once; cut cells integrated
    on a pool of spawned processes, one per host core)."""
    if "d" not in _ORACLE:
        from oracle import discretization as OD
        w = workload_for_bench()
        t0 = time.perf_counter()
        d = OD.from_workload(w, workers=os.cpu_count() or 1)
        _ORACLE.update(d=d, w=w, F=OD.source_vector(d, w.source), setup_s=time.perf_counter() - t0)
    return _ORACLE


def oracle_rate(steps, threads):
    """Oracle CDM loop (Eq. cdm, assembled sparse K, FP64) on the bench workload itself,
    set-up untimed; its mat-vec on ``threads`` host threads.  Returns (DOF-steps/s, s, n_dof)."""
    from oracle import integrators as OI
    o = oracle_disc()
    d, w = o["d"], o["w"]
    t0 = time.perf_counter()
    OI.cdm(d.K, d.ML, 1e-5, steps, F=o["F"], f_e=w.f0, threads=threads)
    el = time.perf_counter() - t0
    return d.n_dof * steps / el, el, d.n_dof


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":")[0].strip().lower()
            if k in ("model name", "cpu part", "hardware"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args, rank, world):
    if rank != 0:
        return
    import torch  # noqa: F401  (launch environment parity)
    cores = os.cpu_count() or 1
    oracle_rate(max(args.warmup, 1), cores)          # set-up and warm-up (untimed)
    rate, el, ndof = oracle_rate(args.steps, cores)
    w = _ORACLE["w"]
    sample = (f"{args.steps} CDM steps of the FP64 oracle (assembled sparse K, mat-vec on {cores} threads) "
              f"on the full {w.name} workload ({ndof} DOFs); set-up untimed ({_ORACLE['setup_s']:.0f} s); "
              f"host CPU: {cpu_model()}")
    line = {"metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": w.name, "grid": list(w.n), "p": w.p,
                       "physics": "plane strain" if w.physics == "elastic" else "scalar wave",
                       "n_dof": ndof, "precision": "fp64 oracle"},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(args, rate=None):
    """Continuous batching of a seeded Poisson stream of mixed 2D/3D requests through the
    batched exact tensor-core path; returns the latency / throughput summary."""
    from paper_2501_19013_gb300 import workloads as W
    from paper_2501_19013_gb300.serve import Request, Server, TcBackend
    n = args.serve_requests
    rate = args.serve_rate if rate is None else rate
    arr = W.poisson_arrivals(n, rate, seed=0)
    reqs = []
    for i in range(n):
        w = W.serving_request(i)
        reqs.append(Request(rid=i, arrival=float(arr[i]), workload=w, steps=w.steps))
    be = TcBackend()
    srv = Server(be, hbm_budget=int(args.serve_budget_gb * (1 << 30)), max_members=args.serve_slots,
                 chunk=32, max_pending=2, workers=8)
    st = srv.run(reqs)
    be.close()
    out = st.summary()
    out.update({"rate_per_s": rate, "hbm_budget_gb": args.serve_budget_gb,
                "slots": args.serve_slots, "precision": "exact",
                "mix": "seeded: 70% 2D plates 32^2-256^2 p2-4 scalar/plane strain with 1-12 holes, "
                       "30% 3D porous cubes 16^3-48^3 p2-3; 500-5000 steps; dt = 0.9 dt_crit each",
                "latency": "arrival -> observer series on the host (includes host setup and dt_crit)"})
    return out


def run_multi_source(args, w, r):
    """Several loads on the benchmark geometry: ``args.sources`` clones of the exact solver
    (shared device geometry and matrices, own state and load), each with an edge traction
    on another window of the left edge, advanced together by the batched exact kernel."""
    from paper_2501_19013_gb300 import ibfem as ib
    S = args.sources
    src = r["solver"]
    clones = [src.clone() for _ in range(S)]
    for k, c in enumerate(clones):
        y0 = 0.05 + 0.7 * k / max(S - 1, 1)
        c.set_source("edge_traction", [y0, y0 + 0.2, 1.0, 0.0], w.f0)
        c.set_initial()
    warm = 64
    n = -(-args.steps // 32) * 32
    b = ib.Batch()
    for c in clones:
        b.add(c, warm + n)
    b.run(warm)
    b.sync()
    t0 = time.perf_counter()
    b.run(n)
    b.sync()
    el = time.perf_counter() - t0
    done = b.poll()
    failed = b.status()[1]
    b.close()
    inf_s, inf_c = src.info(), clones[0].info()
    n_dof = inf_s.n_dof
    out = {"sources": S, "steps": n, "completed": len(done), "failed": failed,
           "dof_steps_per_s": S * n_dof * n / el, "ms_per_batched_step": el * 1e3 / n,
           "single_problem_dof_steps_per_s": n_dof / (r["step_ms"] * 1e-3),
           "device_bytes_fresh_handle": int(inf_s.device_bytes),
           "shared_device_bytes": int(inf_s.shared_device_bytes),
           "device_bytes_per_clone": int(inf_c.device_bytes - inf_c.shared_device_bytes),
           "precision": "exact", "tile_variant": int(inf_c.tile_variant),
           "loads": "edge traction x-direction on x = 0, y in [y0, y0 + 0.2], y0 = 0.05 ... 0.75",
           "timing": "wall clock of ibfem_batch_run + ibfem_batch_sync after 64 warm-up steps; "
                     "the members' states (2 x 8 B x n_dof each) exceed L2"}
    for c in clones:
        c.close()
    return out


def parse_variant(v, w):
    """'fp64' | 'exact' | 'exact64' | 'bf16x3' | 'bf16' -> CDM with the workload's
    stabilisation; 'imex[:exact64|:exact]' -> Newmark IMEX (its explicit part by the FP64, the
    FP64-grade or the exact tensor-core kernel); 'cons[:exact64|:exact]' -> CDM with the
    consistent cut mass; 'ms:<precision>' -> CDM with mass scaling."""
    if v.split(":")[0] == "imex":
        return w.with_(scheme="imex", stab="none"), (v.split(":")[1] if ":" in v else "fp64")
    if v.split(":")[0] == "cons":
        return w.with_(scheme="cdm_consistent"), (v.split(":")[1] if ":" in v else "fp64")
    if v.startswith("ms:"):
        return w.with_(scheme="cdm", stab="mass_scaling"), v[3:]
    return w.with_(scheme="cdm" if w.scheme != "imex" else "cdm",
                   stab=w.stab if w.scheme != "imex" else "mass_scaling"), v


def build_solver(w, precision, stream):
    from paper_2501_19013_gb300 import ibfem as ib
    s = ib.from_workload(w, precision=precision, stream=stream, torch_alloc=True)
    kind, params = ib.source_params(w)
    s.set_source(kind, params, w.f0)
    s.set_observers(w.observers, capacity=w.steps + 1)
    return s


def accuracy_against_fp64(results):
    """Per variant against the FP64 path of the same scheme and stabilisation: the relative
    L2 error of the final field (``rel_l2``) and the paper's observer error (Eq. error:
    e_100 and e_N over all N steps, ``e_obs``); None where there is no comparable FP64 run."""
    from paper_2501_19013_gb300.metrics import observer_errors
    refs = {(r["scheme"], r["stab"]): r for r in results.values() if int(r["info"].precision) == 0}
    for r in results.values():
        r["rel_l2"], r["e_obs"] = None, None
        ref = refs.get((r["scheme"], r["stab"]))
        if ref is None:
            continue
        nr = np.linalg.norm(ref["u_end"])
        r["rel_l2"] = float(np.linalg.norm(r["u_end"] - ref["u_end"]) / nr) if nr > 0 else 0.0
        a, b = r.get("series"), ref.get("series")
        if a is not None and b is not None and a.shape == b.shape and a.shape[0] > 1:
            n = a.shape[0] - 1
            nc = r["info"].ncomp
            e100 = observer_errors(a, b, min(100, n), nc)
            eN = observer_errors(a, b, n, nc)
            r["e_obs"] = {"e_100": e100["mean"], f"e_{n}": eN["mean"], "e_N": eN["mean"],
                          f"e_{n}_per_observer": eN["per_observer"],
                          "observers_left_out": eN["left_out"],
                          "definition": "Eq. error: mean over observers of the relative L2 error "
                                        "of the observer series at n_s equidistant instants, "
                                        "against the FP64 path; observers whose reference norm "
                                        "is below 1e-8 of the largest are left out (counted)"}


def qualifies(r, bar=1e-4):
    """A variant reaches the accuracy bar when both its final-field rel-L2 and its observer
    error e_N against the FP64 path are within it (the FP64 path itself qualifies)."""
    if r["rel_l2"] is None or r["rel_l2"] > bar:
        return False
    return r["e_obs"] is None or r["e_obs"]["e_N"] <= bar


def aggregate_replicas(step_ms, n_dof, world, device=None):
    """Replicas: every rank advances its own copy of the workload.  The job's step time is
    the slowest rank's; the job's throughput counts the DOFs of all ranks."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([step_ms, float(n_dof)], dtype=torch.float64,
                         device=device if device is not None else "cpu")
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = t.clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        return float(mx[0].item()), float(sm[1].item()) / (float(mx[0].item()) * 1e-3)
    return step_ms, n_dof / (step_ms * 1e-3)


# DRAM bytes of one CDM launch (dram__bytes_read.sum + dram__bytes_write.sum, ncu, cold
# cache) of the current kernel code on the benchmark workload (profiles/ gives the command);
# to be re-taken whenever the kernel changes
MEASURED_TRAFFIC = {("op_tc_exact_fused_cdm", "plate_holes_elastic_256x256_p4", 0): 76.364288e6 + 2.137088e6,
                    ("op_tc_exact64_fused_cdm", "plate_holes_elastic_256x256_p4", 0): 51.207424e6 + 0.105984e6}

# arithmetic of each variant's element operator (the state and the update are FP64 in all)
DTYPES = {"fp64": "f64",
          "exact64": "f64-grade: bf16 8-bit slices (7 per operand), exact f32 accumulation, integer assembly, f64 state",
          "exact": "bf16 8-bit slices, exact f32 accumulation, f64 state",
          "bf16x3": "bf16x3, f32 accumulation, f64 state",
          "bf16": "bf16, f32 accumulation, f64 state"}


_FP64_PEAK = {}


def fp64_peak_tflops():
    """FP64 rate of this GPU measured in this run: cuBLAS DGEMM (torch.matmul, 4096^3,
    2 N^3 flop), best of 5 after warm-up, CUDA events."""
    if "v" not in _FP64_PEAK:
        import torch
        n = 4096
        a = torch.randn(n, n, dtype=torch.float64, device="cuda")
        b = torch.randn(n, n, dtype=torch.float64, device="cuda")
        for _ in range(2):
            torch.matmul(a, b)
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        _FP64_PEAK["v"] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
        del a, b
    return _FP64_PEAK["v"]


def algorithmic_bytes(inf, w):
    """Bytes one CDM step must move at FP64 state (the survey's roofline model): 32 B per DOF
    (read u^k, u^{k-1}, dt^2/m; write u^{k+1}), each distinct cut matrix once as packed
    symmetric FP64 (n_loc (n_loc + 1) / 2 entries of 8 B), 4 B of class/index data per cell."""
    n_loc = inf.n_loc
    n_cells = int(np.prod(w.n[:w.dim]))
    return (32.0 * inf.n_dof + 8.0 * inf.n_cut_matrices * n_loc * (n_loc + 1) / 2 + 4.0 * n_cells)


def roofline(prec, kname, kms, inf, w, peaks, r):
    n_dof, n_loc = inf.n_dof, inf.n_loc
    if kname == "imex_solve":
        # the c-set solve of Algorithm 2: both sweeps read L once (FP64 value + 32-bit column
        # index per entry, the survey's 2 nnz(L) x 12 B), plus the residual gather and the
        # correction's c-vectors; bound by its dependency chain, reported against HBM
        nnz = int(inf.nnz_L)
        byts = 2.0 * nnz * 12.0 + 6.0 * 8.0 * int(inf.n_c)
        achieved = byts / (kms * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": kname,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s",
                "algorithmic": f"2 nnz(L) x 12 B (nnz(L) = {nnz}) + 48 B per c-DOF ({int(inf.n_c)}) = {byts:.4e} B",
                "note": "latency-bound: the sweeps follow the dissection tree's dependency chain"}
    if prec == "fp64":
        flops = 2.0 * n_loc * n_loc * inf.n_uncut + 6.0 * n_dof
        achieved = flops / (kms * 1e-3) / 1e12
        peak = fp64_peak_tflops()
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": kname,
                "peak_source": "FP64 cuBLAS DGEMM (4096^3) measured in this run (of measured)",
                "nominal_fp64_tflops": FP64_PEAK_GFLOPS / 1e3,
                "algorithmic": f"2 n_loc^2 per uncut cell + 6 per DOF = {flops:.3e} flop"}
    byts = algorithmic_bytes(inf, w)
    # what this kernel itself moves: FP64 state 24 B/DOF + two FP32 slices of dt^2/m, and
    # the cut matrices as full FP32 (hi, lo) pairs (8 n_loc^2 B per distinct matrix)
    impl = 32.0 * n_dof + 8.0 * inf.n_cut_matrices * n_loc * n_loc + 1.0 * int(np.prod(w.n[:w.dim]))
    achieved = byts / (kms * 1e-3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    variant = r["tile"]["variant"] if r.get("tile") else 0
    traffic = MEASURED_TRAFFIC.get((kname, w.name, variant)) if prec in ("exact", "exact64") else None
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": kname,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback 6.8 TB/s",
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one cold launch of this kernel on this workload" if traffic else None,
            "algorithmic": (f"32 B/DOF ({n_dof}) + packed FP64 cut matrices 4 n_loc (n_loc + 1) B x "
                            f"{inf.n_cut_matrices} + 4 B/cell = {byts:.4e} B"),
            "implementation_bytes": impl,
            "implementation_frac": impl / (kms * 1e-3) / 1e9 / peak}


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2501_19013_gb300 import ibfem as ib

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(dev)          # a real stream: graphs cannot capture the legacy one
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream
    w = workload_for_bench()
    peaks = load_peaks()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    variants = [v for v in args.precisions.split(",") if v]
    results = {}
    dts = {}
    for prec in variants:
        wv, pv = parse_variant(prec, w)
        s = build_solver(wv, pv, sptr)
        info = s.info()
        key = (wv.scheme, wv.stab)
        if key not in dts:
            if args.dt > 0:
                dts[key] = args.dt
            else:
                dt_crit, lam, it = s.crit_dt(max_iter=2000, rtol=1e-7)
                dts[key] = w.dt_factor * dt_crit
        dt = dts[key]
        tile = None
        if pv == "exact" and args.tile_variant >= 0:
            s.set_tile_variant(args.tile_variant)      # fixed tile shape (profiling)
            tile = (args.tile_variant, [float("nan"), float("nan")])
        elif pv == "exact":
            tile = s.autotune(reps=5)      # tile shape of the exact kernel for this problem
        s.set_dt(dt)
        s.set_initial()
        s.step_timed(args.warmup, flush.data_ptr(), FLUSH_BYTES)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = Clocks(local_rank)
        clocks.start()
        t_wall = time.perf_counter()
        ms = s.step_timed(args.steps, flush.data_ptr(), FLUSH_BYTES)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        clk = clocks.stop()
        step_ms = ms.pop("step") / args.steps
        kernels = {k: v / args.steps for k, v in ms.items()}
        # steady state: graph replay back to back (L2-warm), informational
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        steady_ms = e0.elapsed_time(e1) / args.steps
        # accuracy over the configured run (from rest, with the load)
        run_steps = w.steps if args.run_steps < 0 else args.run_steps
        if args.run_time > 0:
            run_steps = int(np.ceil(args.run_time / dt))
        s.set_initial()
        t0 = time.perf_counter()
        s.step(run_steps)
        s.sync()
        run_s = time.perf_counter() - t0
        u_end, _ = s.get_state()
        # observer series of the run (the ring holds w.steps + 1 rows)
        series = s.sample(run_steps + 1) if run_steps <= w.steps else None
        results[prec] = dict(step_ms=step_ms, kernels=kernels, steady_ms=steady_ms, info=info,
                             clocks=clk, run_s=run_s, u_end=u_end, series=series, solver=s, wall=t_wall, dt=dt,
                             run_steps=run_steps, scheme=wv.scheme, stab=wv.stab,
                             tile=None if tile is None else {"variant": tile[0], "cells": list(s.info().tile),
                                                              "ctas_per_sm_cap": int(s.info().tc_ctas_per_sm),
                                                              "autotune_ms_per_apply": [float(x) for x in tile[1]]})
    accuracy_against_fp64(results)
    # headline: fastest variant that reaches rel-L2 <= 1e-4 against FP64
    qual = {p: r for p, r in results.items() if qualifies(r)}
    best = min(qual, key=lambda p: qual[p]["step_ms"]) if qual else variants[0]
    rb = results[best]
    n_dof = rb["info"].n_dof
    step_ms = rb["step_ms"]
    step_ms, value = aggregate_replicas(step_ms, n_dof, world, dev if world > 1 else None)

    # roofline of the dominant kernel
    kname, kms = max(rb["kernels"].items(), key=lambda kv: kv[1])
    inf = rb["info"]
    roof = roofline(parse_variant(best, w)[1], kname, kms, inf, w, peaks, rb)
    for p, r in results.items():
        if p == best:
            r["roofline"] = roof
        else:
            r["roofline"] = roofline(parse_variant(p, w)[1], *max(r["kernels"].items(), key=lambda kv: kv[1]),
                                     r["info"], w, peaks, r)

    # end to end through the C ABI with host buffers
    s = rb["solver"]
    rng = np.random.default_rng(0)
    u0 = np.zeros(n_dof)
    nobs = len(w.observers) * inf.ncomp
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_state(u0, u0, 0)
    s.step(args.steps)
    series = s.sample(args.steps + 1)
    t_e2e = time.perf_counter() - t0
    e2e = {"value": world * n_dof * args.steps / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": 2 * n_dof * 8 / args.steps,
           "d2h_bytes_per_step": series.size * 8 / args.steps,
           "calls": "ibfem_set_state(host) + ibfem_step(K) + ibfem_sample(host)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        oracle_rate(1, cores)                                   # set-up and warm-up (untimed)
        rate, el, nd = oracle_rate(args.cpu_steps, cores)
        rate1, el1, _ = oracle_rate(max(1, args.cpu_steps // 2), 1)
        wo = _ORACLE["w"]
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_steps} CDM steps of the FP64 oracle (assembled sparse K, mat-vec on "
                         f"{cores} threads) on the full {wo.name} workload ({nd} DOFs), set-up untimed "
                         f"({_ORACLE['setup_s']:.0f} s), {el:.1f} s; host CPU: {cpu_model()}",
               "ms_per_step": 1e3 * el / args.cpu_steps,
               "single_core": {"value": rate1, "unit": UNIT, "cores": 1,
                               "ms_per_step": 1e3 * el1 / max(1, args.cpu_steps // 2),
                               "sample": f"{max(1, args.cpu_steps // 2)} steps of the same loop on one thread"},
               "full_run_s_extrapolated": {"all_cores": el / args.cpu_steps * w.steps,
                                           "single_core": el1 / max(1, args.cpu_steps // 2) * w.steps,
                                           "steps": w.steps}}

    variants_out = {}
    for p, r in results.items():
        variants_out[p] = {"dof_steps_per_s": r["info"].n_dof / (r["step_ms"] * 1e-3),
                           "ms_per_step": r["step_ms"], "steady_state_ms_per_step": r["steady_ms"],
                           "rel_l2_vs_fp64_after_run": r["rel_l2"],
                           "observer_error_vs_fp64": r["e_obs"],
                           "run_steps": r["run_steps"], "dt": r["dt"], "scheme": r["scheme"],
                           "stab": r["stab"], "run_wall_s": r["run_s"],
                           "time_to_accuracy_s": (r["step_ms"] * 1e-3 * r["run_steps"]) if qualifies(r) else None,
                           "tile": r.get("tile"),
                           "kernels_ms": r["kernels"], "roofline": r.get("roofline")}
    launches = args.steps * len(rb["kernels"])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES.get(best.split(":")[-1], "f64"), "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.n), "p": w.p,
                       "physics": "plane strain" if w.physics == "elastic" else "scalar wave",
                       "holes": None if w.holes is None else int(len(w.holes)),
                       "voxels": None if w.voxels is None else list(w.voxels.shape),
                       "stab": f"{rb['stab']} eps={w.eps:g} f_lambda={w.f_lambda:g} alpha={w.alpha:g}",
                       "scheme": rb["scheme"],
                       "n_dof": n_dof, "n_uncut": inf.n_uncut, "n_cut": inf.n_cut,
                       "n_cut_matrices": inf.n_cut_matrices,
                       "precision": best, "state": "fp64", "dt": dt,
                       "l2": "flushed before every timed step: 256 MiB device write, then 256 MiB read of another buffer (L2 left holding clean unrelated lines)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": rb["clocks"], "variants": variants_out}
    if rank == 0 and world == 1 and args.sources > 0 and "exact" in results:
        try:
            line["multi_source"] = run_multi_source(args, w, results["exact"])
        except ib.IbfemError as e:          # reported in the line; the headline stands
            line["multi_source"] = {"sources": args.sources, "error": str(e)}
    for r in results.values():
        r["solver"].close()
    if rank == 0 and world == 1 and args.serve_requests > 0:
        line["serving"] = run_serving(args)
        # the same request stream arriving faster: latency and aggregate throughput under load
        loads = []
        for rate in [float(x) for x in args.serve_load_rates.split(",") if x.strip()]:
            o = run_serving(args, rate)
            loads.append({k: o.get(k) for k in ("rate_per_s", "completed", "failed", "p50_s", "p99_s",
                                                 "dof_steps_per_s", "max_concurrent", "p50_stage_s")})
        if loads:
            line["serving_under_load"] = loads
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precisions", default="fp64,exact64,exact")
    ap.add_argument("--cpu-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", type=int, default=256, help="cells per axis of the plate (profiling)")
    ap.add_argument("--dt", type=float, default=0.0, help="fixed dt instead of 0.9 dt_crit (profiling)")
    ap.add_argument("--tile-variant", type=int, default=-1,
                    help="tile shape of the exact kernel instead of the autotuner's choice (profiling)")
    ap.add_argument("--run-steps", type=int, default=-1, help="steps of the accuracy run (-1: the workload's)")
    ap.add_argument("--run-time", type=float, default=0.0, help="simulated time of the accuracy run (overrides steps)")
    ap.add_argument("--sources", type=int, default=8,
                    help="loads of the shared-geometry multi-source run (0: none)")
    ap.add_argument("--serve-requests", type=int, default=48, help="requests of the serving run (0: none)")
    ap.add_argument("--serve-rate", type=float, default=8.0, help="Poisson arrival rate of the serving run (1/s)")
    ap.add_argument("--serve-load-rates", default="16,32",
                    help="further arrival rates (1/s) of the same requests, reported under serving_under_load")
    ap.add_argument("--serve-slots", type=int, default=32, help="maximum concurrent members of the batch")
    ap.add_argument("--serve-budget-gb", type=float, default=64.0, help="device memory budget of the serving run")
    ap.add_argument("--workload", default="plate_holes_elastic",
                    choices=["plate_holes_elastic", "plate_holes_imex", "porous_voxel", "plate_one_hole",
                             "rotated_cube"])
    args = ap.parse_args()
    global GRID, WORKLOAD
    GRID = args.grid
    WORKLOAD = args.workload
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
