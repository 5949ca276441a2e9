"""Seeded synthetic workloads for the Building Cube Method (BCM) time step.

This module only *describes* inputs: cube lists, boundary codes, physical
parameters, body parameters and seeded initial fields.  It holds none of the
method's arithmetic (no stencils, no solid fraction, no solver) so that the CUDA
path and the CPU oracle can both consume it without sharing any numerics.

Grid description (paper section "Building Cube Method"): the domain of each
simulation is covered by equal cubes that are kept in linear arrays holding the
base-corner coordinates, the level (cell size) and, built by each consumer on
its own, the face adjacency.  Every cube has ``B**3`` cells.  Cube corners are
stored in units of the finest cell size of the grid (``h0 / 2**max_level``).
Cubes of one simulation are listed in Z-order (Morton order), the ordering the
paper's mesh generator gives its cubes (section "Data Decomposition").

Boundary codes per domain face, in face order (-x, +x, -y, +y, -z, +z):
  WALL     no-slip wall moving with the face velocity in ``bc_vel`` (lid)
  INFLOW   prescribed inflow velocity ``bc_vel`` (+ optional sine modes)
  SLIP     free slip (zero normal velocity, zero tangential stress)
  OUTFLOW  convective outflow with speed ``uconv``; pressure fixed to 0
  PERIODIC periodic (the opposite face must be PERIODIC as well)
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

WALL, INFLOW, SLIP, OUTFLOW, PERIODIC = 0, 1, 2, 3, 4
BODY_NONE, BODY_SPHERE, BODY_ELLIPSOID = 0, 1, 2
MAX_BODIES = 4
N_MODES = 8

# (k, l) wave numbers of the eight inflow-profile modes in y and z.
INFLOW_MODE_KL = np.array([[1, 1], [1, 2], [2, 1], [2, 2], [1, 3], [3, 1], [2, 3], [3, 2]],
                          dtype=np.int32)


@dataclasses.dataclass
class Body:
    """A rigid body: sphere (radius in axes[0]) or ellipsoid (semi-axes)."""
    kind: int
    center: np.ndarray                  # centre at t = 0
    axes: np.ndarray                    # semi-axes (sphere: axes[0] = radius)
    quat: np.ndarray = dataclasses.field(default_factory=lambda: np.array([1.0, 0, 0, 0]))
    omega: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))
    vel: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))

    def as_row(self) -> np.ndarray:
        """Packed as 17 doubles: kind, c[3], axes[3], q[4], omega[3], vel[3]."""
        return np.concatenate([[float(self.kind)], self.center, self.axes, self.quat,
                               self.omega, self.vel]).astype(np.float64)


@dataclasses.dataclass
class GridSpec:
    """Plain-array description of one or more independent simulations."""
    B: int
    max_level: int
    sim_cube_offset: np.ndarray   # int32 [n_sims+1]
    cube_ijk: np.ndarray          # int32 [n_cubes, 3], finest-cell units
    cube_level: np.ndarray        # int8  [n_cubes]
    sim_extent: np.ndarray        # int32 [n_sims, 3], finest-cell units
    sim_origin: np.ndarray        # f64 [n_sims, 3]
    sim_h0: np.ndarray            # f64 [n_sims] level-0 cell size
    sim_bc: np.ndarray            # int32 [n_sims, 6]
    sim_bc_vel: np.ndarray        # f64 [n_sims, 6, 3]
    sim_nu: np.ndarray            # f64 [n_sims]
    sim_dt: np.ndarray            # f64 [n_sims]
    sim_uconv: np.ndarray         # f64 [n_sims]
    bodies: List[List[Body]]      # per sim
    inflow_modes: np.ndarray      # f64 [n_sims, 8]
    name: str = ""
    steps: int = 1
    rtol: float = 1e-10

    @property
    def n_sims(self) -> int:
        return int(self.sim_cube_offset.shape[0] - 1)

    @property
    def n_cubes(self) -> int:
        return int(self.cube_ijk.shape[0])

    @property
    def n_cells(self) -> int:
        return self.n_cubes * self.B ** 3

    def body_table(self) -> np.ndarray:
        """f64 [n_sims, MAX_BODIES, 17]; unused rows have kind 0."""
        t = np.zeros((self.n_sims, MAX_BODIES, 17))
        for s, bl in enumerate(self.bodies):
            assert len(bl) <= MAX_BODIES
            for b, body in enumerate(bl):
                t[s, b] = body.as_row()
        return t

    def sim_of_cube(self) -> np.ndarray:
        out = np.empty(self.n_cubes, np.int32)
        for s in range(self.n_sims):
            out[self.sim_cube_offset[s]:self.sim_cube_offset[s + 1]] = s
        return out


def _morton_key(ix: int, iy: int, iz: int) -> int:
    key = 0
    for bit in range(21):
        key |= ((ix >> bit) & 1) << (3 * bit)
        key |= ((iy >> bit) & 1) << (3 * bit + 1)
        key |= ((iz >> bit) & 1) << (3 * bit + 2)
    return key


def box_cubes(nx: int, ny: int, nz: int, B: int, level: int = 0, max_level: int = 0,
              offset=(0, 0, 0)) -> np.ndarray:
    """Corners (finest-cell units) of an nx*ny*nz block of level-`level` cubes, Z-ordered."""
    span = B << (max_level - level)
    idx = [(i, j, k) for k in range(nz) for j in range(ny) for i in range(nx)]
    idx.sort(key=lambda t: _morton_key(*t))
    return np.array([[offset[0] + i * span, offset[1] + j * span, offset[2] + k * span]
                     for (i, j, k) in idx], dtype=np.int32).reshape(-1, 3)


def stable_dt(h: float, u_ref: float, nu: float, cfl: float = 0.3, sigma: float = 0.125) -> float:
    """Constant step: the smaller of the convective (CFL) and explicit-diffusion limits."""
    return min(cfl * h / u_ref, sigma * h * h / nu)


def _single(B, cubes, level, max_level, extent, origin, h0, bc, bc_vel, nu, dt, uconv,
            bodies, name, steps, rtol, modes=None) -> GridSpec:
    n = cubes.shape[0]
    return GridSpec(
        B=B, max_level=max_level,
        sim_cube_offset=np.array([0, n], np.int32),
        cube_ijk=np.ascontiguousarray(cubes, dtype=np.int32),
        cube_level=np.ascontiguousarray(level, dtype=np.int8),
        sim_extent=np.array([extent], np.int32),
        sim_origin=np.array([origin], np.float64),
        sim_h0=np.array([h0], np.float64),
        sim_bc=np.array([bc], np.int32),
        sim_bc_vel=np.array([bc_vel], np.float64).reshape(1, 6, 3),
        sim_nu=np.array([nu]), sim_dt=np.array([dt]), sim_uconv=np.array([uconv]),
        bodies=[list(bodies)],
        inflow_modes=np.zeros((1, N_MODES)) if modes is None else np.array([modes], np.float64),
        name=name, steps=steps, rtol=rtol)


def cavity(m: int = 4, B: int = 16, re: float = 100.0, steps: int = 10, rtol: float = 1e-10,
           name: Optional[str] = None) -> GridSpec:
    """Lid-driven cavity on the unit box: m^3 cubes, lid +z moving with u = (1, 0, 0)."""
    n_edge = m * B
    h = 1.0 / n_edge
    nu = 1.0 / re
    bc_vel = np.zeros((6, 3))
    bc_vel[5] = [1.0, 0.0, 0.0]
    return _single(B, box_cubes(m, m, m, B), np.zeros(m ** 3), 0, [n_edge] * 3, [0, 0, 0], h,
                   [WALL] * 6, bc_vel, nu, stable_dt(h, 1.0, nu), 0.0, [],
                   name or f"cavity_{m}x{m}x{m}_B{B}", steps, rtol)


def sphere_channel(nx: int = 16, ny: int = 8, nz: int = 8, B: int = 16, length=(4.0, 2.0, 2.0),
                   radius: float = 0.25, center=(1.0, 1.0, 1.0), re: float = 300.0,
                   steps: int = 200, rtol: float = 1e-8, modes=None,
                   name: Optional[str] = None) -> GridSpec:
    """Uniform inflow U = 1 at -x past a fixed sphere; convective outflow at +x; slip y/z."""
    h = length[0] / (nx * B)
    assert abs(length[1] / (ny * B) - h) < 1e-12 and abs(length[2] / (nz * B) - h) < 1e-12
    nu = 2.0 * radius / re
    bc_vel = np.zeros((6, 3))
    bc_vel[0] = [1.0, 0.0, 0.0]
    body = Body(BODY_SPHERE, np.array(center, np.float64), np.array([radius, radius, radius]))
    return _single(B, box_cubes(nx, ny, nz, B), np.zeros(nx * ny * nz), 0,
                   [nx * B, ny * B, nz * B], [0, 0, 0], h,
                   [INFLOW, OUTFLOW, SLIP, SLIP, SLIP, SLIP], bc_vel, nu,
                   stable_dt(h, 1.0, nu), 1.0, [body],
                   name or f"sphere_{nx}x{ny}x{nz}_B{B}", steps, rtol, modes)


def periodic_box(m: int = 2, B: int = 8, nu: float = 0.01, dt: Optional[float] = None,
                 steps: int = 1, rtol: float = 1e-12) -> GridSpec:
    """All-periodic cube [0, 2pi]^3 with m^3 cubes (Taylor-Green tests)."""
    n_edge = m * B
    h = 2.0 * math.pi / n_edge
    if dt is None:
        dt = stable_dt(h, 1.0, nu)
    return _single(B, box_cubes(m, m, m, B), np.zeros(m ** 3), 0, [n_edge] * 3, [0, 0, 0], h,
                   [PERIODIC] * 6, np.zeros((6, 3)), nu, dt, 0.0, [],
                   f"periodic_{m}_B{B}", steps, rtol)


def concat(specs: List[GridSpec], name: str = "batched") -> GridSpec:
    """Several independent simulations in one flattened cube list (same B, max_level)."""
    B = specs[0].B
    ml = max(s.max_level for s in specs)
    assert all(s.B == B and s.max_level == ml for s in specs)
    offs = [0]
    for s in specs:
        offs.append(offs[-1] + s.n_cubes)
    return GridSpec(
        B=B, max_level=ml,
        sim_cube_offset=np.array(offs, np.int32),
        cube_ijk=np.concatenate([s.cube_ijk for s in specs]).astype(np.int32),
        cube_level=np.concatenate([s.cube_level for s in specs]).astype(np.int8),
        sim_extent=np.concatenate([s.sim_extent for s in specs]).astype(np.int32),
        sim_origin=np.concatenate([s.sim_origin for s in specs]),
        sim_h0=np.concatenate([s.sim_h0 for s in specs]),
        sim_bc=np.concatenate([s.sim_bc for s in specs]).astype(np.int32),
        sim_bc_vel=np.concatenate([s.sim_bc_vel for s in specs]),
        sim_nu=np.concatenate([s.sim_nu for s in specs]),
        sim_dt=np.concatenate([s.sim_dt for s in specs]),
        sim_uconv=np.concatenate([s.sim_uconv for s in specs]),
        bodies=[b for s in specs for b in s.bodies],
        inflow_modes=np.concatenate([s.inflow_modes for s in specs]),
        name=name, steps=specs[0].steps, rtol=specs[0].rtol)


def batched_mix(n_sims: int = 64, seed: int = 0, B: int = 16, lo: int = 8, hi: int = 512,
                steps: int = 50, rtol: float = 1e-8) -> GridSpec:
    """Independent cavity / sphere simulations with log-uniform cube counts in [lo, hi]."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(n_sims):
        n = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        re = rng.uniform(100.0, 1000.0)
        if rng.uniform() < 0.5:
            m = int(min(8, max(2, round(n ** (1.0 / 3.0)))))
            specs.append(cavity(m, B, re, steps, rtol))
        else:
            m = int(max(2, round((n / 2.0) ** (1.0 / 3.0))))
            specs.append(sphere_channel(2 * m, m, m, B, re=re, steps=steps, rtol=rtol))
    return concat(specs, f"batched_{n_sims}_seed{seed}")


# ---------------------------------------------------------------- initial fields

def two_level_cubes(nx: int, ny: int, nz: int, B: int, lo, hi):
    """Level-0 nx*ny*nz cube box whose cubes with index in [lo, hi) are each split
    into eight level-1 cubes (refinement ratio 2).  Corners in level-1 cell units,
    all cubes Z-ordered by corner."""
    span0, span1 = 2 * B, B
    cubes, levels = [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                inside = all(lo[e] <= (i, j, k)[e] < hi[e] for e in range(3))
                if not inside:
                    cubes.append((i * span0, j * span0, k * span0))
                    levels.append(0)
                else:
                    for kk in range(2):
                        for jj in range(2):
                            for ii in range(2):
                                cubes.append((i * span0 + ii * span1, j * span0 + jj * span1,
                                              k * span0 + kk * span1))
                                levels.append(1)
    order = sorted(range(len(cubes)),
                   key=lambda q: _morton_key(*(x // span1 for x in cubes[q])))
    return (np.array([cubes[q] for q in order], np.int32),
            np.array([levels[q] for q in order], np.int8))


def two_level_channel(nx: int = 32, ny: int = 16, nz: int = 16, B: int = 16,
                      lo=(10, 2, 2), hi=(22, 14, 14), h0: float = 1.0 / 64.0,
                      n_bodies: int = 3, seed: int = 0, re: float = 1000.0, steps: int = 100,
                      rtol: float = 1e-8, name: Optional[str] = None) -> GridSpec:
    """Inflow channel on a two-level grid with rotating ellipsoids in the refined block.

    Ellipsoid semi-axes ~ U(0.1, 0.3) (scaled with the box), centres uniform in the
    refined block shrunk by two coarse cells, angular speed ~ U(0.5, 2) rad/s about
    a uniformly random axis, random initial orientation.
    """
    rng = np.random.default_rng(seed)
    cubes, levels = two_level_cubes(nx, ny, nz, B, lo, hi)
    cube_len = B * h0
    scale = cube_len / 0.25          # semi-axes relative to a 0.25-wide coarse cube
    bodies = []
    rmax = 0.0
    for _ in range(n_bodies):
        ax = rng.uniform(0.1, 0.3, 3) * scale
        clo = (np.array(lo) + 2) * cube_len
        chi = (np.array(hi) - 2) * cube_len
        cen = rng.uniform(clo, np.maximum(chi, clo + 1e-9))
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        om = axis * rng.uniform(0.5, 2.0)
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        bodies.append(Body(BODY_ELLIPSOID, cen, ax, q, om, np.zeros(3)))
        rmax = max(rmax, float(np.linalg.norm(om)) * float(ax.max()))
    nu = 1.0 / re
    hf = h0 / 2.0
    bc_vel = np.zeros((6, 3))
    bc_vel[0] = [1.0, 0.0, 0.0]
    ext = [nx * 2 * B, ny * 2 * B, nz * 2 * B]
    return _single(B, cubes, levels, 1, ext, [0, 0, 0], h0,
                   [INFLOW, OUTFLOW, SLIP, SLIP, SLIP, SLIP], bc_vel, nu,
                   stable_dt(hf, 1.0 + rmax, nu), 1.0, bodies,
                   name or f"two_level_{nx}x{ny}x{nz}_B{B}", steps, rtol)


def config_two_level(steps: int = 100) -> GridSpec:
    """20,288 cubes of 16^3 (83.1M cells): 32x16x16 coarse cubes on [0,8]x[0,4]x[0,4],
    the central 12x12x12 coarse cubes refined once; three rotating ellipsoids, Re 1000."""
    return two_level_channel(32, 16, 16, 16, (10, 2, 2), (22, 14, 14), 1.0 / 64.0, 3, 0,
                             1000.0, steps, 1e-8, "two_level_20288cubes_Re1000")


def outflow_slots(spec: GridSpec) -> np.ndarray:
    """(cube, face) pairs that lie on an OUTFLOW domain face, in cube-then-face order.

    Each pair owns a B x B patch of outflow face values (3 components).  This is a
    layout rule only: a face is on the domain boundary when the cube touches the
    low or high end of its simulation's extent along the face normal.
    """
    out = []
    for c in range(spec.n_cubes):
        s = int(np.searchsorted(spec.sim_cube_offset, c, side="right") - 1)
        span = spec.B << (spec.max_level - int(spec.cube_level[c]))
        for f in range(6):
            d, hi = f // 2, f % 2
            on_edge = (spec.cube_ijk[c, d] + span == spec.sim_extent[s, d]) if hi \
                else (spec.cube_ijk[c, d] == 0)
            if on_edge and spec.sim_bc[s, f] == OUTFLOW:
                out.append((c, f))
    return np.array(out, np.int32).reshape(-1, 2)


@dataclasses.dataclass
class State:
    """Cube-major fields, each [n_cubes * B^3] (x fastest inside a cube)."""
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    p: np.ndarray
    ub: np.ndarray   # outflow face values [n_slots, 3, B, B] in outflow_slots() order


def initial_state(spec: GridSpec, seed: int = 0, noise: float = 0.0,
                  base=None) -> State:
    """Zero pressure; velocity = per-sim base velocity + seeded uniform noise.

    ``base`` defaults to the inflow velocity for sims with an INFLOW face and to
    zero otherwise.  Outflow face values start equal to the base velocity.
    """
    rng = np.random.default_rng(seed)
    n = spec.n_cells
    B = spec.B
    u = np.zeros(n)
    v = np.zeros(n)
    w = np.zeros(n)
    slots = outflow_slots(spec)
    ub = np.zeros((slots.shape[0], 3, B, B))
    sim_of = spec.sim_of_cube()
    base_of_sim = np.zeros((spec.n_sims, 3))
    for s in range(spec.n_sims):
        a, b = spec.sim_cube_offset[s] * B ** 3, spec.sim_cube_offset[s + 1] * B ** 3
        if base is not None:
            bv = np.asarray(base, np.float64)
        elif INFLOW in list(spec.sim_bc[s]):
            f = list(spec.sim_bc[s]).index(INFLOW)
            bv = spec.sim_bc_vel[s, f]
        else:
            bv = np.zeros(3)
        base_of_sim[s] = bv
        u[a:b], v[a:b], w[a:b] = bv
    for k, (c, f) in enumerate(slots):
        ub[k] = base_of_sim[sim_of[c]][:, None, None]
    if noise > 0.0:
        u += rng.uniform(-noise, noise, n)
        v += rng.uniform(-noise, noise, n)
        w += rng.uniform(-noise, noise, n)
    return State(u, v, w, np.zeros(n), ub)


@dataclasses.dataclass
class Particles:
    """Lagrangian particles on body surfaces (section "Lagrangian Data Structure"):
    position X at t = 0, the sim and the body (index into that sim's bodies) each one
    belongs to, and its volume weight dV (dc1 dc2 dc3 of Eq. ddeltap)."""
    X: np.ndarray        # f64 [n, 3]
    sim: np.ndarray      # int32 [n]
    body: np.ndarray     # int32 [n]
    dV: np.ndarray       # f64 [n]

    @property
    def n(self) -> int:
        return int(self.X.shape[0])


def surface_particles(spec: GridSpec, sim: int = 0, body: int = 0, spacing: float = 1.0,
                      seed: Optional[int] = None) -> Particles:
    """Particles on the surface of one body at t = 0, about one per surface cell: a
    Fibonacci lattice of N = round(area / (spacing h)^2) points on the unit sphere,
    scaled by the semi-axes and turned by the body's quaternion; weight dV = h^3.
    With a seed the lattice is turned by a seeded random rotation."""
    bd = spec.bodies[sim][body]
    h = float(spec.sim_h0[sim]) / (1 << spec.max_level)
    a, b, c = (float(x) for x in (bd.axes if bd.kind == BODY_ELLIPSOID else
                                  [bd.axes[0]] * 3))
    # Knud Thomsen's approximation of the ellipsoid area (the count only)
    pw = 1.6075
    area = 4 * math.pi * (((a * b) ** pw + (a * c) ** pw + (b * c) ** pw) / 3) ** (1 / pw)
    n = max(1, int(round(area / (spacing * h) ** 2)))
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    th = math.pi * (1.0 + math.sqrt(5.0)) * k
    u = np.stack([r * np.cos(th), r * np.sin(th), z], axis=1)
    if seed is not None:
        q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
        u = u @ q.T
    w, x, y, zq = (float(e) for e in bd.quat)
    R = np.array([[1 - 2 * (y * y + zq * zq), 2 * (x * y - w * zq), 2 * (x * zq + w * y)],
                  [2 * (x * y + w * zq), 1 - 2 * (x * x + zq * zq), 2 * (y * zq - w * x)],
                  [2 * (x * zq - w * y), 2 * (y * zq + w * x), 1 - 2 * (x * x + y * y)]])
    X = (u * np.array([a, b, c])) @ R.T + np.asarray(bd.center, np.float64)
    return Particles(np.ascontiguousarray(X), np.full(n, sim, np.int32),
                     np.full(n, body, np.int32), np.full(n, h ** 3))


def concat_particles(parts: List[Particles]) -> Particles:
    return Particles(np.ascontiguousarray(np.concatenate([p.X for p in parts])),
                     np.concatenate([p.sim for p in parts]).astype(np.int32),
                     np.concatenate([p.body for p in parts]).astype(np.int32),
                     np.concatenate([p.dV for p in parts]))


def config_cavity64(steps: int = 10) -> GridSpec:
    """Lid-driven cavity, 4x4x4 cubes of 16^3, Re 100, FP64, rtol 1e-10."""
    return cavity(4, 16, 100.0, steps, 1e-10, "cavity_64^3_Re100")


def config_sphere(steps: int = 200) -> GridSpec:
    """Sphere R = 0.25 at (1,1,1) in [0,4]x[0,2]x[0,2], 16x8x8 cubes of 16^3, Re 300."""
    return sphere_channel(16, 8, 8, 16, steps=steps, rtol=1e-8, name="sphere_16x8x8_Re300")
