"""Global discretisation: DOF numbering, assembled matrices, loads and observers.

Follows Sec. 2.2: tensor-product GLL Lagrange elements of order p on a uniform Cartesian
grid over the extended domain; fully fictitious cells are dropped (Sec. 3.2); uncut cells
share one reference stiffness (GL rule) and the diagonal GLL mass; cut cells are integrated
by the space tree with alpha^FCM, optionally eigenvalue-stabilised, and lumped by HRZ for
the explicit scheme (Sec. 2.4, 2.5).  The semi-discrete system is M Psi'' + K Psi = F
(Eq. semi); K and the consistent M are *assembled* into sparse matrices here.

DOF numbering: the global node lattice has (n_k p + 1) nodes per axis, lexicographic with
x fastest; nodes belonging to at least one kept cell are numbered in lattice order, and a
node's ncomp DOFs are consecutive (node-major).

Loads (Sec. 3.1, Eq. source_time): a Ricker wavelet f_t(t) = (1 - 2 q^2) exp(-q^2) with
q = pi f_e (t - t_s), t_s = 2 sqrt(6) / (pi f_e), times a spatial vector: a point source
F_i = alpha^FCM(x_s) rho N_i(x_s) (times a direction for elasticity) or an edge traction
F_i = int_Gamma alpha^FCM N_i t ds on the boundary x = lo_x, y in [y0, y1], or the
volumetric Gaussian load of the benchmark (Sec. 3.1), F_i = int alpha^FCM rho f_s N_i dx with
f_s = exp(-|x - x_l|^2 / (2 sigma^2)).

Observers (Sec. 3.2): Psi(x) = sum_j N_j(x) Psi_j in the lowest-numbered kept cell that
contains x.

Pins: the element-by-element K u equals the assembled product, source vectors sum to the
wavelet (partition of unity) and observers interpolate polynomials exactly
(tests/test_oracle_integrators.py); the Gaussian load's integral, centre and alpha
weighting (tests/test_oracle_gauss_load.py); the DOF counts of the paper's rotated cube
(tests/test_oracle_geometry.py); the explicit block of the IMEX partition gives the
paper's IMEX critical time steps for p = 2 to 5 (tests/test_oracle_imex_dt_table.py) and
the assembled consistent mass its consistent-mass ones at p = 2 and 3
(tests/test_timing_table_cpu.py).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import elements as el
from .basis import gauss_legendre, gll_points, lagrange
from .geometry import CUT, OUTSIDE, PHYSICAL, make_geometry
from .quadrature import cut_cell_quadrature, full_cell_quadrature
from .stabilization import evs, hrz, mass_scaling_factor, element_lambda_max


def ricker(t, f_e):
    """Eq. source_time."""
    t_s = 2.0 * math.sqrt(6.0) / (math.pi * f_e)
    q = math.pi * f_e * (t - t_s)
    return (1.0 - 2.0 * q * q) * math.exp(-q * q)


class Discretization:
    def __init__(self, dim, n, p, physics="scalar", geometry=None, alpha=1e-5,
                 quad_depth=3, stab="none", eps=0.0, f_lambda=1e-2, rho=1.0, c=1.0,
                 E=1.0, nu=0.3, lo=None, hi=None, assemble=True, workers=None):
        self.dim = dim
        self.n = np.array(n[:dim], dtype=int)
        self.p = p
        self.physics = physics
        self.ncomp = 2 if physics == "elastic" else 1
        if physics == "elastic" and dim != 2:
            raise ValueError("plane strain is 2D")
        self.geom = geometry
        self.alpha = alpha
        self.quad_depth = quad_depth
        self.stab = stab
        self.eps = eps
        self.f_lambda = f_lambda
        self.rho, self.c, self.E, self.nu = rho, c, E, nu
        self.lo = np.zeros(dim) if lo is None else np.asarray(lo, float)[:dim]
        self.hi = np.ones(dim) if hi is None else np.asarray(hi, float)[:dim]
        self.h = (self.hi - self.lo) / self.n
        self.nn_loc = (p + 1) ** dim
        self.n_loc = self.nn_loc * self.ncomp
        self.lat = self.n * p + 1                     # lattice nodes per axis
        self._classify()
        self._number()
        self._reference_matrices()
        self.K_cut, self.M_cut_cons, self.M_cut_stab, self.ml_cut, self.scale_cut = {}, {}, {}, {}, {}
        self._cut_km = {}
        if assemble:
            if workers and workers > 1 and len(self.cut) > 1:
                self._cut_km = _cut_integrals_in_pool(self, int(workers))
            for e in self.cut:
                self._cut_matrices(e)
            self._cut_km = {}
            self._assemble()

    # ---------------------------------------------------------------- geometry
    def elem_coords(self, e):
        """Element multi-index (x fastest) of flat index e."""
        out = []
        for k in range(self.dim):
            out.append(e % self.n[k])
            e //= self.n[k]
        return np.array(out)

    def elem_box(self, e):
        ij = self.elem_coords(e)
        lo = self.lo + ij * self.h
        return lo, lo + self.h

    def _classify(self):
        ne = int(np.prod(self.n))
        self.cls = np.full(ne, PHYSICAL, dtype=np.int8)
        if self.geom is not None:
            for e in range(ne):
                lo, hi = self.elem_box(e)
                self.cls[e] = self.geom.classify_box(lo, hi)
        self.kept = np.nonzero(self.cls != OUTSIDE)[0]
        self.cut = np.nonzero(self.cls == CUT)[0]
        self.uncut = np.nonzero(self.cls == PHYSICAL)[0]

    # ---------------------------------------------------------------- numbering
    def _lattice_nodes(self, e):
        """Lattice node indices of element e in local (x fastest) order."""
        ij = self.elem_coords(e)
        A = el.local_node_exponents(self.p, self.dim)
        g = ij[None, :] * self.p + A
        idx = np.zeros(len(A), dtype=np.int64)
        stride = 1
        for k in range(self.dim):
            idx += g[:, k] * stride
            stride *= self.lat[k]
        return idx

    def _number(self):
        n_lat = int(np.prod(self.lat))
        used = np.zeros(n_lat, dtype=bool)
        self.elem_lat = {}
        for e in self.kept:
            nodes = self._lattice_nodes(e)
            self.elem_lat[e] = nodes
            used[nodes] = True
        self.node_of_lattice = np.full(n_lat, -1, dtype=np.int64)
        self.lattice_of_node = np.nonzero(used)[0]
        self.node_of_lattice[self.lattice_of_node] = np.arange(len(self.lattice_of_node))
        self.n_nodes = len(self.lattice_of_node)
        self.n_dof = self.n_nodes * self.ncomp
        self.elem_dofs = {}
        for e in self.kept:
            nodes = self.node_of_lattice[self.elem_lat[e]]
            self.elem_dofs[e] = (nodes[:, None] * self.ncomp + np.arange(self.ncomp)[None, :]).ravel()

    # ---------------------------------------------------------------- matrices
    def _matrices(self, lo, hi, X, W, A):
        if self.physics == "elastic":
            return el.elastic_matrices(self.p, lo, hi, X, W, A, self.rho, self.E, self.nu)
        return el.scalar_matrices(self.p, lo, hi, X, W, A, self.rho, self.c)

    def _reference_matrices(self):
        lo0 = self.lo
        hi0 = self.lo + self.h
        X, W, A = full_cell_quadrature(lo0, hi0, self.p)
        self.K_ref, _ = self._matrices(lo0, hi0, X, W, A)
        self.m_gll = el.gll_mass_diagonal(self.p, self.h, self.rho, self.ncomp)
        # M^f of the eigenvalue stabilisation (Sec. 2.5): the mass of a cell lying wholly in
        # Omega as the SCM forms it, with GLL quadrature (Sec. 2.4), hence diagonal
        self.M_full = np.diag(self.m_gll)
        self.lam_ref = element_lambda_max(self.K_ref, self.m_gll)

    def _cut_integrals(self, e):
        """K^e and the consistent M^e of a cut cell by the space-tree quadrature (alpha)."""
        lo, hi = self.elem_box(e)
        X, W, A = cut_cell_quadrature(self.geom, lo, hi, self.p, self.quad_depth, self.alpha)
        return self._matrices(lo, hi, X, W, A)

    def _cut_matrices(self, e):
        """K^e, consistent M^e (alpha), stabilised M^e and the HRZ-lumped diagonal of a
        cut cell (stored in K_cut, M_cut_cons, M_cut_stab, ml_cut, scale_cut)."""
        if e in self._cut_km:
            K, M = self._cut_km[e]
        else:
            K, M = self._cut_integrals(e)
        self.K_cut[e] = K
        self.M_cut_cons[e] = M
        Ms = evs(M, self.M_full, self.eps, self.f_lambda) if self.stab == "evs" else M
        self.M_cut_stab[e] = Ms
        ml = hrz(Ms)
        s = 1.0
        if self.stab == "mass_scaling":
            s = mass_scaling_factor(K, ml, self.lam_ref)
            ml = s * ml
        self.scale_cut[e] = s
        self.ml_cut[e] = ml

    def elem_K(self, e):
        if self.cls[e] == CUT:
            if e not in self.K_cut:
                self._cut_matrices(e)
            return self.K_cut[e]
        return self.K_ref

    def elem_ml(self, e):
        if self.cls[e] == CUT:
            if e not in self.ml_cut:
                self._cut_matrices(e)
            return self.ml_cut[e]
        return self.m_gll

    def cells_of_dof(self, dof):
        """Kept cells whose nodes include the DOF's node (ascending), with local index."""
        node = dof // self.ncomp
        comp = dof % self.ncomp
        lat = self.lattice_of_node[node]
        g = []
        for k in range(self.dim):
            g.append(lat % self.lat[k])
            lat //= self.lat[k]
        out = []
        for offs in np.ndindex(*([2] * self.dim)):
            ij = [g[k] // self.p - offs[k] for k in range(self.dim)]
            if any(ij[k] < 0 or ij[k] >= self.n[k] for k in range(self.dim)):
                continue
            a = [g[k] - ij[k] * self.p for k in range(self.dim)]
            if any(a[k] < 0 or a[k] > self.p for k in range(self.dim)):
                continue
            e = 0
            stride = 1
            for k in range(self.dim):
                e += ij[k] * stride
                stride *= self.n[k]
            if self.cls[e] == OUTSIDE:
                continue
            loc = 0
            stride = 1
            for k in range(self.dim):
                loc += a[k] * stride
                stride *= self.p + 1
            out.append((e, loc * self.ncomp + comp))
        return sorted(set(out))

    def local_cdm_update(self, dofs, u, u_prev, dt, fk=None):
        """Eq. cdm evaluated at selected DOFs only, from element contributions of the
        cells that contain them (no assembly): u_i^{k+1} for i in dofs."""
        out = np.zeros(len(dofs))
        for n_, i in enumerate(dofs):
            ku = 0.0
            m = 0.0
            for e, loc in self.cells_of_dof(i):
                D = self.elem_dofs[e]
                ku += self.elem_K(e)[loc] @ u[D]
                m += self.elem_ml(e)[loc]
            f = 0.0 if fk is None else fk[n_]
            out[n_] = 2.0 * u[i] - u_prev[i] + dt * dt / m * (f - ku)
        return out

    def _assemble(self):
        rows, cols, vals = [], [], []
        ml = np.zeros(self.n_dof)
        ii, jj = np.meshgrid(np.arange(self.n_loc), np.arange(self.n_loc), indexing="ij")
        ii, jj = ii.ravel(), jj.ravel()
        # uncut cells: one shared reference matrix
        if len(self.uncut):
            D = np.stack([self.elem_dofs[e] for e in self.uncut])      # (nu, n_loc)
            rows.append(D[:, ii].ravel())
            cols.append(D[:, jj].ravel())
            vals.append(np.tile(self.K_ref.ravel(), len(self.uncut)))
            np.add.at(ml, D.ravel(), np.tile(self.m_gll, len(self.uncut)))
        for e in self.cut:
            D = self.elem_dofs[e]
            rows.append(D[ii])
            cols.append(D[jj])
            vals.append(self.K_cut[e].ravel())
            np.add.at(ml, D, self.ml_cut[e])
        r = np.concatenate(rows) if rows else np.zeros(0, int)
        cc = np.concatenate(cols) if cols else np.zeros(0, int)
        v = np.concatenate(vals) if vals else np.zeros(0)
        self.K = sp.csr_matrix((v, (r, cc)), shape=(self.n_dof, self.n_dof))
        self.ML = ml

    def consistent_mass(self, stabilised=False):
        """Global mass with GLL diagonal for uncut cells and the consistent cut mass."""
        rows, cols, vals = [], [], []
        diag = np.zeros(self.n_dof)
        for e in self.uncut:
            np.add.at(diag, self.elem_dofs[e], self.m_gll)
        for e in self.cut:
            D = self.elem_dofs[e]
            Mc = self.M_cut_stab[e] if stabilised else self.M_cut_cons[e]
            rows.append(np.repeat(D, len(D)))
            cols.append(np.tile(D, len(D)))
            vals.append(Mc.ravel())
        M = sp.diags(diag).tocsr()
        if rows:
            M = M + sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                  shape=(self.n_dof, self.n_dof))
        return M

    # ---------------------------------------------------------------- element-by-element K u
    def apply_K_elementwise(self, u):
        """Brute-force check helper: K u = sum_e P_e^T K^e P_e u without assembly."""
        out = np.zeros_like(u)
        for e in self.kept:
            D = self.elem_dofs[e]
            out[D] += self.elem_K(e) @ u[D]
        return out

    # ---------------------------------------------------------------- points
    def locate(self, x):
        """Lowest-numbered kept element containing x (closed boxes)."""
        x = np.asarray(x, float)
        ij = np.floor((x - self.lo) / self.h).astype(int)
        cands = []
        for offs in np.ndindex(*([2] * self.dim)):
            c = ij - np.array(offs)
            if np.all(c >= 0) and np.all(c < self.n):
                lo = self.lo + c * self.h
                if np.all(x >= lo - 1e-14) and np.all(x <= lo + self.h + 1e-14):
                    e = 0
                    stride = 1
                    for k in range(self.dim):
                        e += c[k] * stride
                        stride *= self.n[k]
                    if self.cls[e] != OUTSIDE:
                        cands.append(e)
        if not cands:
            raise ValueError(f"point {x} is not in a kept element")
        return min(cands)

    def point_weights(self, x):
        e = self.locate(x)
        lo, hi = self.elem_box(e)
        N, _ = el.shape_functions(self.p, lo, hi, np.asarray(x, float)[None, :])
        return e, N[0]

    def point_load(self, x, direction=None):
        """Spatial vector of a point source at x (Sec. 3.1 volumetric source, point form)."""
        e, N = self.point_weights(x)
        a = 1.0
        if self.geom is not None and not self.geom.in_physical(np.asarray(x, float)[None, :])[0]:
            a = self.alpha
        F = np.zeros(self.n_dof)
        nodes = self.node_of_lattice[self.elem_lat[e]]
        if self.ncomp == 1:
            F[nodes] += a * self.rho * N
        else:
            d = np.asarray(direction if direction is not None else [1.0, 0.0], float)
            for c in range(self.ncomp):
                F[nodes * self.ncomp + c] += a * self.rho * N * d[c]
        return F

    def edge_traction_load(self, y0, y1, t):
        """int over {x = lo_x, y in [y0, y1]} of alpha^FCM N_i t ds (2D)."""
        assert self.dim == 2
        t = np.atleast_1d(np.asarray(t, float))
        F = np.zeros(self.n_dof)
        xg, wg = gauss_legendre(self.p + 1)
        for ey in range(self.n[1]):
            e = ey * self.n[0]
            if self.cls[e] == OUTSIDE:
                continue
            lo, hi = self.elem_box(e)
            a0, a1 = max(lo[1], y0), min(hi[1], y1)
            if a1 <= a0:
                continue
            ys = a0 + (xg + 1.0) * 0.5 * (a1 - a0)
            ws = wg * 0.5 * (a1 - a0)
            X = np.stack([np.full_like(ys, lo[0]), ys], axis=1)
            N, _ = el.shape_functions(self.p, lo, hi, X)
            A = np.ones(len(ys)) if self.geom is None else np.where(self.geom.in_physical(X), 1.0, self.alpha)
            integ = (ws * A) @ N          # (nn,)
            nodes = self.node_of_lattice[self.elem_lat[e]]
            for c in range(self.ncomp):
                F[nodes * self.ncomp + c] += integ * t[c if len(t) > c else 0]
        return F

    def gauss_load(self, x_l, sigma):
        """F_i = int over the kept cells of alpha^FCM rho f_s N_i, f_s the Gaussian of Sec. 3.1
        (weak form Eq. weak_form_extended, load term).

        Quadrature (the paper does not give one; reading shared with the library): every
        kept cell whose box lies within 8 sigma of x_l is split into m^d equal subcells,
        m = max(1, ceil(max_k h_k / sigma)), each integrated with (p + 4)^d Gauss-Legendre
        points, alpha^FCM evaluated at the points.  Beyond 8 sigma f_s < 1.3e-14."""
        x_l = np.asarray(x_l, dtype=np.float64)
        reach = 8.0 * sigma
        m = max(1, int(math.ceil(float(np.max(self.h)) / sigma)))
        xg, wg = gauss_legendre(self.p + 4)
        F = np.zeros(self.n_dof)
        for e in range(int(np.prod(self.n))):
            if self.cls[e] == OUTSIDE:
                continue
            lo, hi = self.elem_box(e)
            gap = np.maximum(np.maximum(lo - x_l, x_l - hi), 0.0)
            if np.sqrt(np.sum(gap * gap)) > reach:
                continue
            # composite 1D rules per axis (m subintervals), then the tensor grid
            pts, wts = [], []
            for k in range(self.dim):
                a = lo[k] + (hi[k] - lo[k]) * np.arange(m) / m
                b = lo[k] + (hi[k] - lo[k]) * np.arange(1, m + 1) / m
                pts.append((a[:, None] + (xg[None, :] + 1.0) * 0.5 * (b - a)[:, None]).ravel())
                wts.append((np.repeat(0.5 * (b - a), len(xg)) * np.tile(wg, m)))
            grids = np.meshgrid(*pts, indexing="ij")
            X = np.stack([g.ravel() for g in grids], axis=1)
            Wg = np.meshgrid(*wts, indexing="ij")
            Wq = np.prod(np.stack([g.ravel() for g in Wg], axis=1), axis=1)
            A = np.ones(len(X)) if self.geom is None else np.where(self.geom.in_physical(X), 1.0, self.alpha)
            f = np.exp(-0.5 * np.sum((X - x_l[None, :]) ** 2, axis=1) / (sigma * sigma))
            N, _ = el.shape_functions(self.p, lo, hi, X)
            integ = (Wq * A * f * self.rho) @ N
            nodes = self.node_of_lattice[self.elem_lat[e]]
            for c in range(self.ncomp):
                F[nodes * self.ncomp + c] += integ
        return F

    def observer_matrix(self, pts):
        """Sparse (n_obs * ncomp, n_dof) interpolation: row o*ncomp + c samples comp c."""
        rows, cols, vals = [], [], []
        for o, x in enumerate(np.atleast_2d(pts)):
            e, N = self.point_weights(x)
            nodes = self.node_of_lattice[self.elem_lat[e]]
            for c in range(self.ncomp):
                rows.append(np.full(len(nodes), o * self.ncomp + c))
                cols.append(nodes * self.ncomp + c)
                vals.append(N)
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(len(np.atleast_2d(pts)) * self.ncomp, self.n_dof))

    # ---------------------------------------------------------------- IMEX partition
    def explicit_block(self):
        """(K_dd, M_L on d, d indices): the explicit block of the IMEX partition (Sec. 2.6).
        A d-DOF has support in uncut cells only, so its rows of K and of the lumped mass
        are sums of the reference stiffness and the GLL mass of those cells; no cut-cell
        integral is needed."""
        c = np.zeros(self.n_dof, dtype=bool)
        c[self.c_dofs()] = True
        nl = self.n_loc
        ii, jj = np.meshgrid(np.arange(nl), np.arange(nl), indexing="ij")
        D = np.stack([self.elem_dofs[e] for e in self.uncut])
        K = sp.csr_matrix((np.tile(self.K_ref.ravel(), len(self.uncut)),
                           (D[:, ii.ravel()].ravel(), D[:, jj.ravel()].ravel())),
                          shape=(self.n_dof, self.n_dof))
        ml = np.zeros(self.n_dof)
        np.add.at(ml, D.ravel(), np.tile(self.m_gll, len(self.uncut)))
        d = np.nonzero(~c)[0]
        return K[d][:, d], ml[d], d

    def c_dofs(self, all_dofs=False):
        """DOFs with support in at least one cut cell (Sec. 2.6)."""
        if all_dofs:
            return np.arange(self.n_dof)
        mark = np.zeros(self.n_dof, dtype=bool)
        for e in self.cut:
            mark[self.elem_dofs[e]] = True
        return np.nonzero(mark)[0]


def _cut_integrals_of(args):
    disc, cells = args
    return {e: disc._cut_integrals(e) for e in cells}


def _cut_integrals_in_pool(disc, workers):
    """The cut cells' K^e, M^e (the same function per cell as the serial loop) on a pool of
    spawned processes; only the work is split, every cell's arithmetic is unchanged."""
    import multiprocessing as mp
    cells = [int(e) for e in disc.cut]
    n = max(1, min(workers, len(cells)))
    chunks = [cells[i::n] for i in range(n)]
    out = {}
    with mp.get_context("spawn").Pool(n) as pool:
        for res in pool.map(_cut_integrals_of, [(disc, c) for c in chunks]):
            out.update(res)
    return out


def from_workload(w, **over):
    """Build a Discretization for a ``workloads.Workload``."""
    geom = make_geometry(w.dim, holes=w.holes, voxels=w.voxels, lo=w.lo, hi=w.hi,
                         rotated_box=getattr(w, "rotated_box", None))
    kw = dict(dim=w.dim, n=w.n, p=w.p, physics=w.physics, geometry=geom, alpha=w.alpha,
              quad_depth=w.quad_depth, stab=w.stab, eps=w.eps, f_lambda=w.f_lambda,
              rho=w.rho, c=w.c, E=w.E, nu=w.nu, lo=w.lo, hi=w.hi)
    kw.update(over)
    return Discretization(**kw)


def source_vector(disc, src):
    kind = src.get("kind", "point")
    if kind == "point":
        return disc.point_load(np.asarray(src["x"], float), src.get("dir"))
    if kind == "edge_traction":
        return disc.edge_traction_load(src["y0"], src["y1"], src.get("t", [1.0, 0.0]))
    if kind == "gauss":
        return disc.gauss_load(np.asarray(src["x"], float), float(src["sigma"]))
    raise ValueError(kind)
