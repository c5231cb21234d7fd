"""Thin ctypes binding of ``libibfem.so`` (argument marshalling only).

Every function below forwards to the C entry point of the same name declared in
``include/ibfem.h``; all arithmetic runs in the library's CUDA kernels and host setup.
The binding raises ``IbfemError`` on a negative status and ``ImportError`` when the
shared library has not been built -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libibfem.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_DIVERGED, ERR_TIMEOUT, ERR_GEOMETRY, ERR_EIG, ERR_STATE = 0, -1, -2, -3, -4, -5, -6, -7, -8
GEOM_NONE, GEOM_HOLES, GEOM_VOXELS, GEOM_ROTATED_BOX = 0, 1, 2, 3
STAB_NONE, STAB_EVS, STAB_MASS_SCALING = 0, 1, 2
SCALAR, ELASTIC_PLANE_STRAIN = 0, 1
CDM, IMEX, CDM_CONSISTENT = 0, 1, 2
SCHEMES = {"cdm": CDM, "imex": IMEX, "cdm_consistent": CDM_CONSISTENT}
FP64, EXACT_TC, BF16X3_TC, BF16_TC, EXACT64_TC = 0, 1, 2, 3, 4
SRC_NONE, SRC_POINT, SRC_EDGE_TRACTION, SRC_GAUSS = 0, 1, 2, 3

PRECISIONS = {"fp64": FP64, "exact": EXACT_TC, "bf16x3": BF16X3_TC, "bf16": BF16_TC, "exact64": EXACT64_TC}


class IbfemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ibfem error {code}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class Geometry(C.Structure):
    _fields_ = [("kind", C.c_int), ("count", C.c_int), ("shapes", C.POINTER(C.c_double)),
                ("voxels", C.POINTER(C.c_uint8)), ("vn", C.c_int * 3), ("quad_depth", C.c_int)]


class Stab(C.Structure):
    _fields_ = [("kind", C.c_int), ("eps", C.c_double), ("f_lambda", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Options(C.Structure):
    _fields_ = [("physics", C.c_int), ("rho", C.c_double), ("c", C.c_double), ("E", C.c_double),
                ("nu", C.c_double), ("scheme", C.c_int), ("precision", C.c_int),
                ("stream", C.c_void_p), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("device", C.c_int), ("host_only", C.c_int)]


class Info(C.Structure):
    _fields_ = [("n_dof", C.c_int64), ("n_lattice_dof", C.c_int64), ("n_elem", C.c_int64),
                ("n_uncut", C.c_int64), ("n_cut", C.c_int64), ("n_outside", C.c_int64),
                ("n_c", C.c_int64), ("nnz_L", C.c_int64), ("n_levels", C.c_int32),
                ("n_loc", C.c_int32), ("ncomp", C.c_int32), ("precision", C.c_int32),
                ("step", C.c_int64), ("t", C.c_double), ("dt", C.c_double),
                ("lambda_ref", C.c_double), ("device_bytes", C.c_size_t),
                ("n_cut_matrices", C.c_int64), ("tile_variant", C.c_int32), ("tile", C.c_int32 * 3),
                ("shared_device_bytes", C.c_size_t), ("tc_ctas_per_sm", C.c_int32),
                ("autotune_cached", C.c_int32)]


_lib = None
DP = C.POINTER(C.c_double)


def lib():
    """Load the shared library (raises ImportError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built: run __graft_entry__.build() first")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    sig = {
        "ibfem_create": (C.c_int, [C.POINTER(Grid), C.c_int, C.POINTER(Geometry), C.c_double,
                                   C.POINTER(Stab), C.POINTER(Options), C.POINTER(vp)]),
        "ibfem_destroy": (C.c_int, [vp]),
        "ibfem_last_error": (C.c_char_p, []),
        "ibfem_info": (C.c_int, [vp, C.POINTER(Info)]),
        "ibfem_set_source": (C.c_int, [vp, C.c_int, DP, C.c_int, C.c_double]),
        "ibfem_set_observers": (C.c_int, [vp, C.c_int, DP, C.c_int64]),
        "ibfem_set_initial": (C.c_int, [vp, DP, DP]),
        "ibfem_crit_dt": (C.c_int, [vp, C.c_int, C.c_double, DP, DP, C.POINTER(C.c_int)]),
        "ibfem_set_dt": (C.c_int, [vp, C.c_double]),
        "ibfem_step": (C.c_int, [vp, C.c_int64]),
        "ibfem_sync": (C.c_int, [vp]),
        "ibfem_check_bounded_wait": (C.c_int, [vp, C.c_int]),
        "ibfem_check_solve_schedule": (C.c_int, [vp, C.c_double, C.c_uint64, C.POINTER(C.c_int64),
                                                 C.POINTER(C.c_double)]),
        "ibfem_step_timed": (C.c_int, [vp, C.c_int64, vp, C.c_size_t, DP, C.c_int, C.POINTER(C.c_int)]),
        "ibfem_kernel_name": (C.c_char_p, [vp, C.c_int]),
        "ibfem_sample": (C.c_int, [vp, C.c_int64, DP, C.POINTER(C.c_int64)]),
        "ibfem_get_state": (C.c_int, [vp, DP, DP]),
        "ibfem_set_state": (C.c_int, [vp, DP, DP, C.c_int64]),
        "ibfem_apply_operator": (C.c_int, [vp, DP, DP]),
        "ibfem_get_lumped_mass": (C.c_int, [vp, DP]),
        "ibfem_get_cut_cells": (C.c_int, [vp, C.POINTER(C.c_int64)]),
        "ibfem_get_element": (C.c_int, [vp, C.c_int64, DP, DP]),
        "ibfem_get_element_mass": (C.c_int, [vp, C.c_int64, DP]),
        "ibfem_apply_operator_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                                   vp, vp, vp, C.c_int64, vp, vp, vp, vp, vp]),
        "ibfem_upload": (C.c_int, [vp]),
        "ibfem_clone": (C.c_int, [vp, C.POINTER(vp)]),
        "ibfem_set_tile_variant": (C.c_int, [vp, C.c_int]),
        "ibfem_autotune": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int), DP]),
        "ibfem_batch_create": (C.c_int, [vp, C.c_int, C.POINTER(vp)]),
        "ibfem_batch_add": (C.c_int, [vp, vp, C.c_int64]),
        "ibfem_batch_run": (C.c_int, [vp, C.c_int64]),
        "ibfem_batch_poll": (C.c_int, [vp, C.POINTER(vp), C.c_int, C.POINTER(C.c_int)]),
        "ibfem_batch_status": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
        "ibfem_batch_sync": (C.c_int, [vp]),
        "ibfem_batch_wait": (C.c_int, [vp, C.c_int]),
        "ibfem_batch_destroy": (C.c_int, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc):
    if rc != OK:
        raise IbfemError(rc, lib().ibfem_last_error().decode())


def _dp(a):
    return None if a is None else a.ctypes.data_as(DP)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class Solver:
    """One simulation handle (``ibfem_t``)."""

    def __init__(self, dim, n, p, *, lo=None, hi=None, physics="scalar", rho=1.0, c=1.0,
                 E=1.0, nu=0.3, alpha=1e-5, holes=None, voxels=None, rotated_box=None,
                 quad_depth=3, stab="none", eps=0.0, f_lambda=1e-2, scheme="cdm",
                 precision="fp64", stream=None, device=0, host_only=False, torch_alloc=False,
                 allocator=None):
        L = lib()
        g = Grid()
        g.dim = dim
        for k in range(3):
            g.n[k] = int(n[k]) if k < dim else 1
            g.lo[k] = (lo[k] if lo is not None else 0.0) if k < dim else 0.0
            g.hi[k] = (hi[k] if hi is not None else 1.0) if k < dim else 1.0
        geo = Geometry()
        self._keep = []
        geo.quad_depth = quad_depth
        if holes is not None and len(holes):
            hs = _f64(np.asarray(holes).reshape(-1))
            self._keep.append(hs)
            geo.kind, geo.count, geo.shapes = GEOM_HOLES, len(holes), _dp(hs)
        elif voxels is not None:
            vx = np.ascontiguousarray(voxels, dtype=np.uint8)   # [z, y, x] or [y, x]
            self._keep.append(vx)
            geo.kind = GEOM_VOXELS
            geo.voxels = vx.ctypes.data_as(C.POINTER(C.c_uint8))
            shp = vx.shape[::-1]
            for k in range(3):
                geo.vn[k] = shp[k] if k < len(shp) else 1
        elif rotated_box is not None:
            rb = _f64(rotated_box)
            self._keep.append(rb)
            geo.kind, geo.shapes = GEOM_ROTATED_BOX, _dp(rb)
        st = Stab()
        st.kind = {"none": STAB_NONE, "evs": STAB_EVS, "mass_scaling": STAB_MASS_SCALING}[stab]
        st.eps, st.f_lambda = eps, f_lambda
        o = Options()
        o.physics = SCALAR if physics == "scalar" else ELASTIC_PLANE_STRAIN
        o.rho, o.c, o.E, o.nu = rho, c, E, nu
        o.scheme = SCHEMES[scheme]
        o.precision = PRECISIONS[precision]
        o.stream = stream
        o.device = device
        o.host_only = 1 if host_only else 0
        if torch_alloc and allocator is None:
            import torch
            dev = device

            def _talloc(nbytes):
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev)

            allocator = (_talloc, torch.cuda.caching_allocator_delete)
        if allocator is not None:
            # ``allocator`` = (alloc(nbytes) -> device address or None, free(address)): the
            # library's dev_alloc / dev_free callbacks (a None or an exception is a failure)
            a_fn, f_fn = allocator

            def _alloc(nbytes, ctx):
                try:
                    return a_fn(int(nbytes))
                except Exception:
                    return None

            def _free(ptr, ctx):
                f_fn(ptr)

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
            o.dev_alloc, o.dev_free = self._alloc_cb, self._free_cb
        h = C.c_void_p()
        _check(L.ibfem_create(C.byref(g), p, C.byref(geo), alpha, C.byref(st), C.byref(o), C.byref(h)))
        self.h = h
        self.dim = dim
        inf = self.info()
        self.n_dof = inf.n_dof
        self.ncomp = inf.ncomp
        self.n_loc = inf.n_loc

    # -- lifetime
    def close(self):
        if getattr(self, "h", None):
            lib().ibfem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls
    def upload(self):
        """Move a host-only handle onto its device (``ibfem_upload``)."""
        _check(lib().ibfem_upload(self.h))

    def clone(self):
        """A new solver on this discretisation (``ibfem_clone``): shares the device geometry
        and matrices, owns its state, load, observers and dt (initially this one's)."""
        h = C.c_void_p()
        _check(lib().ibfem_clone(self.h, C.byref(h)))
        c = Solver.__new__(Solver)
        c.h = h
        c.dim, c.n_dof, c.ncomp, c.n_loc = self.dim, self.n_dof, self.ncomp, self.n_loc
        c._keep = []
        for k in ("_alloc_cb", "_free_cb"):   # the clone may free shared arrays through them
            if hasattr(self, k):
                setattr(c, k, getattr(self, k))
        return c

    def set_tile_variant(self, variant):
        _check(lib().ibfem_set_tile_variant(self.h, int(variant)))

    def autotune(self, reps=5):
        """Time both tile shapes and keep the faster: (variant, [ms variant 0, ms variant 1])."""
        v = C.c_int()
        ms = np.zeros(2)
        _check(lib().ibfem_autotune(self.h, int(reps), C.byref(v), _dp(ms)))
        return v.value, ms

    def info(self):
        i = Info()
        _check(lib().ibfem_info(self.h, C.byref(i)))
        return i

    def set_source(self, kind, params, f_e):
        k = {"none": SRC_NONE, "point": SRC_POINT, "edge_traction": SRC_EDGE_TRACTION, "gauss": SRC_GAUSS}[kind]
        pr = _f64(params) if params is not None else np.zeros(1)
        _check(lib().ibfem_set_source(self.h, k, _dp(pr), len(pr) if params is not None else 0, f_e))

    def set_observers(self, pts, capacity):
        pts = _f64(np.asarray(pts).reshape(-1))
        self.n_obs = len(pts) // self.dim
        _check(lib().ibfem_set_observers(self.h, self.n_obs, _dp(pts), int(capacity)))

    def set_dt(self, dt):
        _check(lib().ibfem_set_dt(self.h, float(dt)))

    def set_initial(self, u0=None, v0=None):
        u0, v0 = _f64(u0), _f64(v0)
        _check(lib().ibfem_set_initial(self.h, _dp(u0), _dp(v0)))

    def crit_dt(self, max_iter=500, rtol=1e-10):
        dt, lam, it = C.c_double(), C.c_double(), C.c_int()
        _check(lib().ibfem_crit_dt(self.h, max_iter, rtol, C.byref(dt), C.byref(lam), C.byref(it)))
        return dt.value, lam.value, it.value

    def step(self, n):
        _check(lib().ibfem_step(self.h, int(n)))

    def step_timed(self, n, flush_ptr=None, flush_bytes=0):
        """Run n steps with per-kernel CUDA events (optionally writing ``flush_bytes`` at
        device address ``flush_ptr`` before each step); returns {slot name: total ms},
        slot "step" being whole steps."""
        ms = np.zeros(8)
        ns = C.c_int()
        _check(lib().ibfem_step_timed(self.h, int(n), flush_ptr, int(flush_bytes), _dp(ms), 8,
                                      C.byref(ns)))
        return {lib().ibfem_kernel_name(self.h, i).decode(): ms[i] for i in range(ns.value)}

    def sync(self):
        _check(lib().ibfem_sync(self.h))

    def check_bounded_wait(self, polls):
        """Enqueue one bounded wait that runs out (``ibfem_check_bounded_wait``)."""
        _check(lib().ibfem_check_bounded_wait(self.h, int(polls)))

    def check_solve_schedule(self, beta_dt2=0.0, seed=0):
        """Host check of the GPU block solve's schedule (``ibfem_check_solve_schedule``):
        returns (violations, larger relative error of the two sweeps against substitution)."""
        v = C.c_int64()
        e = C.c_double()
        _check(lib().ibfem_check_solve_schedule(self.h, float(beta_dt2), int(seed), C.byref(v), C.byref(e)))
        return int(v.value), float(e.value)

    def sample(self, max_rows):
        nr = self.n_obs * self.ncomp
        out = np.zeros((int(max_rows), max(nr, 1)))
        rows = C.c_int64()
        _check(lib().ibfem_sample(self.h, int(max_rows), _dp(out), C.byref(rows)))
        return out[: rows.value, :nr]

    def get_state(self):
        u = np.zeros(self.n_dof)
        up = np.zeros(self.n_dof)
        _check(lib().ibfem_get_state(self.h, _dp(u), _dp(up)))
        return u, up

    def set_state(self, u, u_prev, step):
        u, up = _f64(u), _f64(u_prev)
        _check(lib().ibfem_set_state(self.h, _dp(u), _dp(up), int(step)))

    def apply_operator(self, x):
        x = _f64(x)
        y = np.zeros(self.n_dof)
        _check(lib().ibfem_apply_operator(self.h, _dp(x), _dp(y)))
        return y

    def lumped_mass(self):
        m = np.zeros(self.n_dof)
        _check(lib().ibfem_get_lumped_mass(self.h, _dp(m)))
        return m

    def cut_cells(self):
        n = self.info().n_cut
        out = np.zeros(max(n, 1), dtype=np.int64)
        _check(lib().ibfem_get_cut_cells(self.h, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return out[:n]

    def element(self, cell):
        K = np.zeros((self.n_loc, self.n_loc))
        ml = np.zeros(self.n_loc)
        _check(lib().ibfem_get_element(self.h, int(cell), _dp(K), _dp(ml)))
        return K, ml


    def element_mass(self, cell):
        """Consistent element mass of the consistent-mass schemes (``ibfem_get_element_mass``)."""
        M = np.zeros((self.n_loc, self.n_loc))
        _check(lib().ibfem_get_element_mass(self.h, int(cell), _dp(M)))
        return M


class Batch:
    """Continuous batching of exact tensor-core CDM solvers (``ibfem_batch_*``)."""

    def __init__(self, stream=None, device=0):
        b = C.c_void_p()
        _check(lib().ibfem_batch_create(stream, device, C.byref(b)))
        self.b = b
        self._members = {}   # handle address -> Solver

    def add(self, solver, n_steps):
        _check(lib().ibfem_batch_add(self.b, solver.h, int(n_steps)))
        self._members[solver.h.value] = solver

    def run(self, n):
        _check(lib().ibfem_batch_run(self.b, int(n)))

    def poll(self, max_done=64):
        """Solvers whose budget is used up (ordinary handles again)."""
        arr = (C.c_void_p * max(int(max_done), 1))()
        n = C.c_int()
        _check(lib().ibfem_batch_poll(self.b, arr, int(max_done), C.byref(n)))
        return [self._members.pop(arr[i]) for i in range(n.value)]

    def status(self):
        a, f, s = C.c_int(), C.c_int(), C.c_int64()
        _check(lib().ibfem_batch_status(self.b, C.byref(a), C.byref(f), C.byref(s)))
        return a.value, f.value, s.value

    def wait(self, max_pending):
        _check(lib().ibfem_batch_wait(self.b, int(max_pending)))

    def sync(self):
        _check(lib().ibfem_batch_sync(self.b))

    def close(self):
        if getattr(self, "b", None):
            lib().ibfem_batch_destroy(self.b)
            self.b = None
            self._members = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def apply_operator_noalloc(dim, p, ncomp, n_cells, cell_class, cut_index, cut_cells, n_cut,
                           K_ref, K_cut, x, y, stream=None):
    """Forward to ``ibfem_apply_operator_noalloc``; every array argument is a device address
    (int), ``stream`` a cudaStream_t handle (int) or None."""
    nc = (C.c_int * 3)(*[int(v) for v in list(n_cells) + [1] * (3 - len(n_cells))])
    _check(lib().ibfem_apply_operator_noalloc(dim, p, ncomp, nc, cell_class, cut_index, cut_cells,
                                              int(n_cut), K_ref, K_cut, x, y, stream))


def from_workload(w, precision="fp64", host_only=False, scheme=None, **kw):
    """Create a Solver for a ``workloads.Workload`` (geometry and material only)."""
    return Solver(w.dim, w.n, w.p, lo=w.lo, hi=w.hi, physics=w.physics, rho=w.rho, c=w.c,
                  E=w.E, nu=w.nu, alpha=w.alpha, holes=w.holes, voxels=w.voxels,
                  rotated_box=getattr(w, "rotated_box", None),
                  quad_depth=w.quad_depth, stab=w.stab, eps=w.eps, f_lambda=w.f_lambda,
                  scheme=scheme or w.scheme, precision=precision, host_only=host_only, **kw)


def source_params(w):
    s = w.source
    if s.get("kind", "point") == "point":
        return "point", list(s["x"]) + list(s.get("dir", []))
    if s["kind"] == "gauss":
        return "gauss", list(s["x"]) + [s["sigma"]]
    return "edge_traction", [s["y0"], s["y1"]] + list(s.get("t", [1.0, 0.0]))
