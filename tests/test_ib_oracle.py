"""Pins of the oracle's Lagrangian-particle immersed boundary (R19 in oracle/bcm_oracle.c)
to things other than itself: the values and moments of the 3-point delta, exact
interpolation of linear fields, conservation and adjointness of spreading, the weights
of a particle at a cell centre and at a cell corner worked out by hand, a body moving
with a uniform flow as a fixed point, the fluid momentum an impulsively moved body
imparts in a periodic box, and the closed-form position update of a rotating body."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1808_04099_gb300 import workloads as W


def test_delta3_values_and_moments():
    d = O.Oracle.delta3
    # the printed piecewise function worked out at its nodes by hand
    for r, v in ((0.0, 0.75), (0.5, 0.5), (-0.5, 0.5), (1.0, 0.125), (-1.0, 0.125),
                 (1.5, 0.0), (-1.5, 0.0), (2.0, 0.0), (0.25, 0.6875), (1.25, 0.03125)):
        assert d(r) == pytest.approx(v, abs=1e-15), r
    # continuity at the joints, partition of unity and zero first moment (the
    # conditions the function is built to satisfy, not its formula)
    for x in (0.5, 1.5):
        assert abs(d(x - 1e-12) - d(x + 1e-12)) < 1e-11
    for r in np.linspace(0.0, 1.0, 41):
        w = [d(r - j) for j in range(-2, 3)]
        assert sum(w) == pytest.approx(1.0, abs=1e-15)
        assert sum((r - j) * wj for j, wj in zip(range(-2, 3), w)) == pytest.approx(0.0, abs=1e-15)


def _centres(spec):
    """Cell-centre coordinates of every cell, from the cube corners and h alone."""
    B = spec.B
    h = spec.sim_h0[0]
    i = (np.arange(B) + 0.5)
    cc = np.asarray(spec.cube_ijk, np.float64).reshape(-1, 1, 1, 1, 3)
    k3, j3, i3 = np.meshgrid(i, i, i, indexing="ij")
    off = np.stack([i3, j3, k3], axis=-1)[None]
    x = spec.sim_origin[0] + h * (cc + off)
    return x.reshape(-1, 3)


def _grid():
    return W.sphere_channel(4, 2, 2, 8, length=(2.0, 1.0, 1.0), radius=0.2,
                            center=(0.9, 0.5, 0.45))


def test_interpolation_reproduces_linear_fields():
    spec = _grid()
    o = O.Oracle(spec)
    parts = W.surface_particles(spec, seed=3)
    x = _centres(spec)
    rng = np.random.default_rng(0)
    for _ in range(3):
        a, b = rng.standard_normal(), rng.standard_normal(3)
        f = a + x @ b
        U = o.ib_interpolate(f, parts)
        ref = a + parts.X @ b
        assert np.abs(U - ref).max() <= 1e-13 * (1 + np.abs(ref).max())


def test_spread_conserves_and_is_the_adjoint_of_interpolation():
    spec = _grid()
    o = O.Oracle(spec)
    parts = W.surface_particles(spec, seed=4)
    h = spec.sim_h0[0]
    rng = np.random.default_rng(1)
    F = rng.standard_normal(parts.n)
    f = o.ib_spread(F, parts)
    assert f.sum() * h ** 3 == pytest.approx((F * parts.dV).sum(), rel=1e-13)
    u = rng.standard_normal(spec.n_cells)
    lhs = (F * o.ib_interpolate(u, parts) * parts.dV).sum()
    rhs = (u * f).sum() * h ** 3
    assert lhs == pytest.approx(rhs, rel=1e-12)


def _one(spec, X):
    return W.Particles(np.ascontiguousarray(np.asarray(X, np.float64).reshape(1, 3)),
                       np.zeros(1, np.int32), np.zeros(1, np.int32),
                       np.array([spec.sim_h0[0] ** 3]))


def test_single_particle_weights_by_hand():
    spec = _grid()
    o = O.Oracle(spec)
    h = spec.sim_h0[0]
    x = _centres(spec)
    c = np.array([0.9, 0.5, 0.45])
    # a particle on a cell centre: weights (3/4 or 1/8) per axis, 27 cells
    centre = x[np.argmin(((x - c) ** 2).sum(1))]
    f = o.ib_spread(np.ones(1), _one(spec, centre))
    d = np.rint(np.abs(x - centre) / h).astype(int)
    near = (d <= 1).all(1)
    want = np.where(d == 0, 0.75, 0.125).prod(1)
    assert np.abs(f[near] - want[near]).max() <= 1e-15 and np.abs(f[~near]).max() == 0.0
    assert near.sum() == 27
    # a particle on a cell corner: 1/2 per axis on the 8 cells around it, 0 elsewhere
    corner = centre + 0.5 * h
    f = o.ib_spread(np.ones(1), _one(spec, corner))
    dd = np.abs(x - corner) / h
    eight = (np.abs(dd - 0.5) < 1e-9).all(1)
    assert eight.sum() == 8
    assert np.abs(f[eight] - 0.125).max() <= 1e-15 and np.abs(f[~eight]).max() <= 1e-15


def _periodic_with_body(vel=(0.0, 0.0, 0.0), omega=(0.0, 0.0, 0.0)):
    """Periodic box of 16^3 cells, a sphere of radius L/5 at its centre (its particles
    stay more than two cells away from the domain faces)."""
    spec = W.periodic_box(2, 8, nu=0.01)
    L = spec.sim_extent[0] * spec.sim_h0[0]
    spec.bodies[0] = [W.Body(W.BODY_SPHERE, L / 2, np.array([L[0] / 5] * 3),
                             omega=np.array(omega, np.float64), vel=np.array(vel, np.float64))]
    return spec


def _state(spec, U):
    st = O.Oracle(spec).new_state(W.initial_state(spec))
    for e, k in enumerate("uvw"):
        st[k][:] = U[e]
    st["p"][:] = 0.0
    return st


def test_comoving_body_is_a_fixed_point():
    U = np.array([0.3, -0.2, 0.1])
    spec = _periodic_with_body(vel=U)
    o = O.Oracle(spec)
    parts = W.surface_particles(spec, seed=5)
    X = parts.X.copy()
    st = _state(spec, U)
    stats, rc, F = o.step_particles(st, X, parts, nsteps=3, rtol=1e-13)
    assert rc == 0
    for e, k in enumerate("uvw"):
        assert np.abs(st[k] - U[e]).max() <= 1e-13
    assert np.abs(F).max() <= 1e-11 and np.abs(stats[0]["drag"]).max() <= 1e-13
    assert np.abs(X - (parts.X + 3 * spec.sim_dt[0] * U)).max() <= 1e-14


def test_impulsive_body_imparts_its_momentum():
    """Fluid at rest in a periodic box, body set moving with v: every particle sees
    F = v / dt; the projection keeps the total momentum of a periodic box, so after one
    step the fluid carries sum_p F_p dV_p dt = N dV v, and the drag is -N dV v / dt."""
    v = np.array([0.4, 0.1, -0.25])
    spec = _periodic_with_body(vel=v)
    o = O.Oracle(spec)
    parts = W.surface_particles(spec, seed=6)
    X = parts.X.copy()
    st = _state(spec, np.zeros(3))
    dt, h = spec.sim_dt[0], spec.sim_h0[0]
    stats, rc, F = o.step_particles(st, X, parts, nsteps=1, rtol=1e-13)
    assert rc == 0
    assert np.abs(F - v / dt).max() <= 1e-12 * np.abs(v / dt).max()
    total = parts.n * parts.dV[0] * v
    mom = np.array([st[k].sum() * h ** 3 for k in "uvw"])
    assert np.abs(mom - total).max() <= 1e-12 * np.abs(total).max()
    assert np.abs(np.array(stats[0]["drag"]) + total / dt).max() <= 1e-12 * np.abs(total / dt).max()


def test_rotating_body_moves_its_particles_rigidly():
    om = np.array([0.0, 0.0, 2.0])
    spec = _periodic_with_body(omega=om)
    o = O.Oracle(spec)
    parts = W.surface_particles(spec, seed=7)
    X = parts.X.copy()
    st = _state(spec, np.zeros(3))
    dt = spec.sim_dt[0]
    o.step_particles(st, X, parts, nsteps=1, rtol=1e-12)
    c = spec.sim_extent[0] * spec.sim_h0[0] / 2
    want = parts.X + dt * np.cross(om, parts.X - c)
    assert np.abs(X - want).max() <= 1e-15
    # the body velocity at the particles is the rigid motion, and the step's radius
    # grows by the explicit update only: |X - c|^2 (1 + (|omega| dt)^2) in the plane
    r0 = np.hypot(*(parts.X - c)[:, :2].T)
    r1 = np.hypot(*(X - c)[:, :2].T)
    assert np.abs(r1 - r0 * math.sqrt(1 + (2.0 * dt) ** 2)).max() <= 1e-14


def test_no_particles_is_the_body_free_step():
    spec = _periodic_with_body()
    st0 = W.initial_state(spec, seed=9, noise=1e-2)
    o = O.Oracle(spec)
    a = o.new_state(st0)
    empty = W.Particles(np.zeros((0, 3)), np.zeros(0, np.int32), np.zeros(0, np.int32),
                        np.zeros(0))
    o.step_particles(a, np.zeros((0, 3)), empty, nsteps=2, rtol=1e-12)
    spec.bodies[0] = []
    o2 = O.Oracle(spec)
    b = o2.new_state(st0)
    o2.step(b, nsteps=2, rtol=1e-12)
    for k in "uvwp":
        assert np.array_equal(a[k], b[k]), k
