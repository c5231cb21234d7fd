"""Seeded synthetic inputs shared by the CUDA library, the oracle, the tests and the bench.

This module only *generates inputs*: hole lists, voxel images, source and observer
positions, and the named workload configurations.  It contains none of the solver's
arithmetic (no basis functions, quadrature, matrices or time stepping), so that the
oracle and the CUDA path stay independent and both can be fed the same arrays.

Randomness comes from SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then the two
xor-shift-multiply mixing rounds; doubles take the top 53 bits.

Workloads (all on the unit square / cube, Neumann boundaries):

* ``plate_one_hole`` - 2D scalar wave, one circular hole r=0.2 at the centre,
  16x16 elements, p=2, alpha=1e-5, quadtree depth 3, Ricker point source f0=5.
* ``plate_holes_elastic`` - 2D plane-strain elastodynamics (E=1, nu=0.3, rho=1),
  12 seeded holes r in [0.02, 0.08], 256x256 elements, p=4, eigenvalue
  stabilisation (f_lambda=1e-2, eps=1e-4, alpha=1e-12), Ricker edge traction, 10k steps.
* ``plate_holes_imex`` - 2D scalar wave on the same holes, 512x512, p=3, IMEX
  (alpha=1e-12) against explicit with mass scaling.
* ``porous_voxel`` - 3D scalar wave, 128^3 voxel image of random spherical voids
  at >=30 % porosity, 64^3 elements, p=3, alpha=1e-5, eigenvalue stabilisation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (Steele et al. 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))


def random_holes(count: int, r_min: float, r_max: float, seed: int,
                 edge_margin: float = 0.02, gap: float = 0.01,
                 max_tries: int = 100000) -> np.ndarray:
    """Non-overlapping circles in the unit square by rejection sampling.

    Each circle keeps ``r + edge_margin`` from the square's edges and a gap of at
    least ``gap`` to every other circle.  Returns ``(count, 3)`` rows ``(cx, cy, r)``.
    """
    rng = SplitMix64(seed)
    out = []
    tries = 0
    while len(out) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random_holes: could not place all holes")
        r = rng.uniform(r_min, r_max)
        m = r + edge_margin
        cx = rng.uniform(m, 1.0 - m)
        cy = rng.uniform(m, 1.0 - m)
        ok = True
        for (ox, oy, orr) in out:
            if math.hypot(cx - ox, cy - oy) < r + orr + gap:
                ok = False
                break
        if ok:
            out.append((cx, cy, r))
    return np.array(out, dtype=np.float64)


def random_void_image(vn: int, r_min: float, r_max: float, porosity: float,
                      seed: int, max_spheres: int = 100000) -> np.ndarray:
    """Voxel image ``(vn, vn, vn)`` uint8, index order [z, y, x], 1 = void.

    Spheres with radius uniform in ``[r_min, r_max]`` voxels and centres uniform in
    the voxel box are carved (voxel centre strictly inside a sphere -> void) until
    the void fraction reaches ``porosity``.
    """
    rng = SplitMix64(seed)
    img = np.zeros((vn, vn, vn), dtype=np.uint8)
    c = np.arange(vn, dtype=np.float64) + 0.5
    target = porosity * vn ** 3
    nvoid = 0
    for _ in range(max_spheres):
        if nvoid >= target:
            break
        r = rng.uniform(r_min, r_max)
        cx = rng.uniform(0.0, vn)
        cy = rng.uniform(0.0, vn)
        cz = rng.uniform(0.0, vn)
        lo = [max(0, int(math.floor(q - r))) for q in (cz, cy, cx)]
        hi = [min(vn, int(math.ceil(q + r)) + 1) for q in (cz, cy, cx)]
        zz = c[lo[0]:hi[0]][:, None, None]
        yy = c[lo[1]:hi[1]][None, :, None]
        xx = c[lo[2]:hi[2]][None, None, :]
        inside = (xx - cx) ** 2 + (yy - cy) ** 2 + (zz - cz) ** 2 < r * r
        sub = img[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
        nvoid += int(np.count_nonzero(inside & (sub == 0)))
        sub[inside] = 1
    return img


def nearest_solid_point(img: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Centre of the solid voxel nearest to ``x`` (unit-cube coordinates)."""
    vn = img.shape[0]
    solid = np.argwhere(img == 0)  # rows (z, y, x)
    centres = (solid[:, ::-1].astype(np.float64) + 0.5) / vn
    d = np.sum((centres - x[None, :]) ** 2, axis=1)
    return centres[int(np.argmin(d))]


@dataclass
class Workload:
    """A named synthetic problem: grid, discretisation, geometry, source, steps."""
    name: str
    dim: int
    n: tuple
    p: int
    physics: str                      # "scalar" or "elastic"
    rho: float = 1.0
    c: float = 1.0
    E: float = 1.0
    nu: float = 0.3
    alpha: float = 1e-5
    quad_depth: int = 3
    holes: Optional[np.ndarray] = None   # (k, d+1) rows (centre..., r)
    voxels: Optional[np.ndarray] = None  # uint8 [z, y, x], 1 = void
    rotated_box: Optional[np.ndarray] = None  # (edge, centre[3], T[9] row-major): x = c + T x' 
    stab: str = "none"                # "none" | "evs" | "mass_scaling"
    eps: float = 0.0
    f_lambda: float = 1e-2
    scheme: str = "cdm"               # "cdm" | "imex"
    source: dict = field(default_factory=dict)
    f0: float = 5.0
    steps: int = 200
    dt_factor: float = 0.9
    observers: Optional[np.ndarray] = None
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def default_observers(dim: int) -> np.ndarray:
    if dim == 2:
        return np.array([[0.25, 0.25], [0.75, 0.25], [0.25, 0.75], [0.75, 0.75],
                         [0.5, 0.9], [0.9, 0.5]], dtype=np.float64)
    return np.array([[0.25, 0.25, 0.25], [0.75, 0.75, 0.75], [0.5, 0.5, 0.9],
                     [0.9, 0.5, 0.5]], dtype=np.float64)


def near_load_observers() -> np.ndarray:
    """Observers of the plate benchmark within the reach of its wave: the edge traction on
    x = 0, y in [0.4, 0.6] with a Ricker pulse of f_e = 10 (delay 0.156) sends a P wave at
    c_p = 1.16 (E = 1, nu = 0.3, rho = 1) about 0.3 into the plate in 10 000 steps of
    4.2e-5, so every point here is passed by the pulse during the run."""
    return np.array([[0.05, 0.5], [0.1, 0.42], [0.1, 0.58], [0.2, 0.5], [0.06, 0.32],
                     [0.2, 0.64]], dtype=np.float64)


def observers_outside_holes(pts: np.ndarray, holes: Optional[np.ndarray]) -> np.ndarray:
    """Move observer points that fall inside a hole radially to 1.05 r from its centre."""
    pts = np.array(pts, dtype=np.float64)
    if holes is None:
        return pts
    d = pts.shape[1]
    for i in range(len(pts)):
        for row in holes:
            c, r = row[:d], row[d]
            v = pts[i] - c
            dist = float(np.sqrt(np.sum(v * v)))
            if dist < r * 1.05:
                if dist == 0.0:
                    v = np.zeros(d)
                    v[0] = 1.0
                    dist = 1.0
                pts[i] = c + v / dist * r * 1.05
    return pts


def plate_one_hole() -> Workload:
    return Workload(name="plate_one_hole_16x16_p2", dim=2, n=(16, 16), p=2,
                    physics="scalar", alpha=1e-5, quad_depth=3,
                    holes=np.array([[0.5, 0.5, 0.2]]), stab="none",
                    source={"kind": "point", "x": [0.15, 0.5]}, f0=5.0, steps=200,
                    observers=default_observers(2))


def plate_holes_elastic(n: int = 256, p: int = 4, count: int = 12, seed: int = 0,
                        steps: int = 10000) -> Workload:
    holes = random_holes(count, 0.02, 0.08, seed)
    return Workload(name=f"plate_holes_elastic_{n}x{n}_p{p}", dim=2, n=(n, n), p=p,
                    physics="elastic", E=1.0, nu=0.3, rho=1.0, alpha=1e-12,
                    quad_depth=3, holes=holes, stab="evs", eps=1e-4, f_lambda=1e-2,
                    source={"kind": "edge_traction", "y0": 0.4, "y1": 0.6,
                            "t": [1.0, 0.0]},
                    f0=10.0, steps=steps, observers=observers_outside_holes(near_load_observers(), holes))


def plate_holes_imex(n: int = 512, p: int = 3, count: int = 12, seed: int = 0,
                     steps: int = 1000, scheme: str = "imex") -> Workload:
    holes = random_holes(count, 0.02, 0.08, seed)
    return Workload(name=f"plate_holes_{scheme}_{n}x{n}_p{p}", dim=2, n=(n, n), p=p,
                    physics="scalar", alpha=1e-12, quad_depth=3, holes=holes,
                    stab="none" if scheme == "imex" else "mass_scaling",
                    scheme=scheme, source={"kind": "point", "x": [0.1, 0.5]},
                    f0=10.0, steps=steps, observers=observers_outside_holes(default_observers(2), holes))


def porous_voxel(n: int = 64, vn: int = 128, p: int = 3, seed: int = 0,
                 steps: int = 2000, porosity: float = 0.30) -> Workload:
    img = random_void_image(vn, 4.0 * vn / 128.0, 12.0 * vn / 128.0, porosity, seed)
    xs = nearest_solid_point(img, np.array([0.1, 0.5, 0.5]))
    obs = np.array([nearest_solid_point(img, x) for x in default_observers(3)])
    return Workload(name=f"porous_voxel_{n}^3_p{p}", dim=3, n=(n, n, n), p=p,
                    physics="scalar", alpha=1e-5, quad_depth=1, voxels=img,
                    stab="evs", eps=1e-4, f_lambda=1e-2,
                    source={"kind": "point", "x": list(xs)}, f0=10.0, steps=steps,
                    observers=obs)


def _solid_point(rng: SplitMix64, dim: int, holes: Optional[np.ndarray], img: Optional[np.ndarray]) -> np.ndarray:
    """A point in [0.1, 0.9]^dim outside every hole (2D) or moved to solid voxels (3D)."""
    for _ in range(1000):
        x = np.array([rng.uniform(0.1, 0.9) for _ in range(dim)])
        if img is not None:
            return nearest_solid_point(img, x)
        if holes is None or all(np.sum((x - h[:dim]) ** 2) > (1.1 * h[dim]) ** 2 for h in holes):
            return x
    raise RuntimeError("no solid point found")


def serving_request(seed: int) -> Workload:
    """One request of the serving stream: a random 2D plate with holes (32^2 to 256^2 cells,
    p = 2..4, scalar or plane strain) or a random 3D porous cube (16^3 to 48^3 cells,
    p = 2..3, voxel image at 2 voxels per cell and axis), eigenvalue stabilisation, a
    Ricker point source at a random solid position and 500 to 5000 steps."""
    rng = SplitMix64(0x5EB1CE ^ (seed * 0x9E3779B97F4A7C15))

    def pick(values, weights):
        u, acc = rng.uniform(), 0.0
        for v, w in zip(values, weights):
            acc += w
            if u < acc:
                return v
        return values[-1]

    steps = 500 + int(rng.uniform() * 4501)
    if rng.uniform() < 0.7:
        n = pick([32, 64, 128, 256], [0.35, 0.3, 0.2, 0.15])
        p = pick([2, 3, 4], [1 / 3, 1 / 3, 1 / 3])
        physics = "elastic" if rng.uniform() < 0.3 else "scalar"
        count = 1 + int(rng.uniform() * 12)
        holes = random_holes(count, 0.02, 0.08, seed=int(rng.next_u64() & 0xFFFFFFFF))
        xs = _solid_point(rng, 2, holes, None)
        src = {"kind": "point", "x": list(xs)}
        if physics == "elastic":
            src["dir"] = [1.0, 0.0]
        return Workload(name=f"serve_{seed}_2d_{n}_p{p}_{physics}", dim=2, n=(n, n), p=p,
                        physics=physics, alpha=1e-5, quad_depth=3, holes=holes, stab="evs",
                        eps=1e-4, f_lambda=1e-2, source=src, f0=10.0, steps=steps,
                        observers=observers_outside_holes(default_observers(2), holes))
    n = pick([16, 24, 32, 48], [0.4, 0.3, 0.2, 0.1])
    p = pick([2, 3], [0.5, 0.5])
    vn = 2 * n
    img = random_void_image(vn, max(1.0, 4.0 * vn / 128.0), max(2.0, 12.0 * vn / 128.0),
                            0.1 + 0.2 * rng.uniform(), int(rng.next_u64() & 0xFFFFFFFF))
    xs = _solid_point(rng, 3, None, img)
    obs = np.array([nearest_solid_point(img, x) for x in default_observers(3)])
    return Workload(name=f"serve_{seed}_3d_{n}_p{p}", dim=3, n=(n, n, n), p=p, physics="scalar",
                    alpha=1e-5, quad_depth=1, voxels=img, stab="evs", eps=1e-4, f_lambda=1e-2,
                    source={"kind": "point", "x": list(xs)}, f0=10.0, steps=steps, observers=obs)


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: exponential gaps of mean 1 / rate."""
    rng = SplitMix64(0xA5517A1 ^ seed)
    t, out = 0.0, np.zeros(count)
    for i in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate
        out[i] = t
    return out


def rotation_zyx(phi: float, theta: float, psi: float) -> np.ndarray:
    """Rotation of the cube's local frame, Cardan angles (radians) taken as intrinsic
    rotations about z, then y, then x: T = R_z(phi) R_y(theta) R_x(psi)."""
    cz, sz = math.cos(phi), math.sin(phi)
    cy, sy = math.cos(theta), math.sin(theta)
    cx, sx = math.cos(psi), math.sin(psi)
    Rz = np.array([[cz, -sz, 0.0], [sz, cz, 0.0], [0.0, 0.0, 1.0]])
    Ry = np.array([[cy, 0.0, sy], [0.0, 1.0, 0.0], [-sy, 0.0, cy]])
    Rx = np.array([[1.0, 0.0, 0.0], [0.0, cx, -sx], [0.0, sx, cx]])
    return Rz @ Ry @ Rx


def rotated_cube(ne: int = 13, p: int = 3, alpha: float = 1e-12, stab: str = "evs",
                 eps: float = 1e-4, quad_depth: Optional[int] = None, steps: int = 2000) -> Workload:
    """The paper's benchmark (Sec. 3.1): a cube of edge 0.3 rotated by the Cardan angles
    (10, 10, 10) degrees about the centre of the extended cube [0, 0.5]^3, scalar wave
    (rho = c = 1), a Gaussian volumetric load (sigma = 0.01) centred on one face of the
    cube times a Ricker wavelet (f_e = 10), and the 11 observers of the paper's table of
    observer locations (source, centre, face, 4 edge centres, 4 corners).  The quadtree
    depth of the cut cells defaults to p + 1, which reproduces the paper's critical time
    steps of the consistent-mass CDM."""
    if quad_depth is None:
        quad_depth = p + 1
    lp, le = 0.3, 0.5
    T = rotation_zyx(*(math.radians(10.0),) * 3)
    c = np.full(3, le / 2.0)
    xs = c + T @ np.array([-lp / 2.0, 0.0, 0.0])
    # observer table in the cube's corner-based local frame [0, l]^3, then centred
    loc = [(0.0, 0.5, 0.5), (0.5, 0.5, 0.5), (1.0, 0.5, 0.5)]
    loc += [(0.5, 0.5 + a, 0.5 + b) for a in (-0.5, 0.5) for b in (-0.5, 0.5)]
    loc += [(1.0, 0.5 + a, 0.5 + b) for a in (-0.5, 0.5) for b in (-0.5, 0.5)]
    obs = np.array([c + T @ ((np.array(q) - 0.5) * lp) for q in loc])
    # corners and edges lie on the immersed boundary: pull them 1e-9 into the cube
    obs = np.array([c + (x - c) * (1.0 - 1e-9) for x in obs])
    return Workload(name=f"rotated_cube_{ne}^3_p{p}", dim=3, n=(ne, ne, ne), p=p,
                    physics="scalar", alpha=alpha, quad_depth=quad_depth,
                    rotated_box=np.concatenate([[lp], c, T.ravel()]), stab=stab, eps=eps,
                    f_lambda=1e-2, source={"kind": "gauss", "x": list(xs), "sigma": 0.01},
                    f0=10.0, steps=steps, observers=obs, hi=(le, le, le))


WORKLOADS = {
    "plate_one_hole": plate_one_hole,
    "plate_holes_elastic": plate_holes_elastic,
    "plate_holes_imex": plate_holes_imex,
    "porous_voxel": porous_voxel,
    "rotated_cube": rotated_cube,
}
