"""The Lagrangian-particle immersed boundary on the GPU (bcm_set_particles) against the
oracle (R19 in oracle/bcm_oracle.c): interpolation and spreading of seeded fields at
seeded particles, the per-cube sets, whole steps with fixed and moving bodies in FP64
(1e-10) and mixed precision (1e-6), graph-captured steps, and the full-size sphere
flow.  Both sides use the same particles from workloads.surface_particles."""
import numpy as np
import pytest

import oracle as O
from paper_1808_04099_gb300 import workloads as W
from _util import demean_per_sim, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1808_04099_gb300 import bcm  # noqa: E402

TOL64, TOL32 = 1e-10, 1e-6


def sphere(B=8, nx=4, ny=2, nz=2, **kw):
    L = nx / ny
    return W.sphere_channel(nx, ny, nz, B, length=(L, 1.0, nz / ny), radius=0.2,
                            center=(0.8, 0.5, 0.45 * nz / ny), **kw)


def moving_box():
    """Periodic box with a translating, rotating ellipsoid and a uniform flow."""
    spec = W.periodic_box(2, 8, nu=0.02)
    L = spec.sim_extent[0] * spec.sim_h0[0]
    q = np.array([np.cos(0.3), np.sin(0.3) / np.sqrt(3), np.sin(0.3) / np.sqrt(3),
                  np.sin(0.3) / np.sqrt(3)])
    spec.bodies[0] = [W.Body(W.BODY_ELLIPSOID, L / 2, np.array([L[0] / 5, L[0] / 7, L[0] / 6]),
                             quat=q, omega=np.array([0.0, 0.3, 1.1]),
                             vel=np.array([0.2, -0.1, 0.05]))]
    return spec


GRIDS = {
    "sphere_B8": lambda: sphere(8),
    "sphere_B16": lambda: W.sphere_channel(2, 1, 1, 16, length=(2.0, 1.0, 1.0), radius=0.2,
                                           center=(0.6, 0.5, 0.5)),
    "moving_box": moving_box,
}


@pytest.mark.parametrize("name", sorted(GRIDS))
def test_interpolation_and_spreading_match_oracle(name):
    spec = GRIDS[name]()
    parts = W.surface_particles(spec, seed=11)
    o = O.Oracle(spec)
    g = bcm.Grid(spec, bcm.PREC_F64)
    g.set_particles(parts)
    rng = np.random.default_rng(12)
    f = rng.standard_normal(spec.n_cells)
    U = g.ib_interpolate(f).cpu().numpy()
    assert np.abs(U - o.ib_interpolate(f, parts)).max() <= 1e-13 * np.abs(f).max()
    F = rng.standard_normal(parts.n)
    s = g.ib_spread(F).cpu().numpy()
    ref = o.ib_spread(F, parts)
    assert np.abs(s - ref).max() <= 1e-13 * np.abs(ref).max()


def expected_sets(spec, X):
    """Cube of every particle from its position (host): the cube whose cells contain
    the particle's cell, -1 outside."""
    B, h = spec.B, spec.sim_h0[0]
    I = np.floor((X - spec.sim_origin[0]) / h).astype(int)
    where = {tuple(spec.cube_ijk[c] // B): c for c in range(spec.n_cubes)}
    return np.array([where.get(tuple(i // B), -1) for i in I])


def check_sets(g, spec, X):
    start, ids = g.particle_sets()
    cube = expected_sets(spec, X)
    assert start[0] == 0 and start[-1] == (cube >= 0).sum()
    assert np.all(np.diff(start) >= 0)
    got = np.full(len(X), -1)
    for c in range(spec.n_cubes):
        members = ids[start[c]:start[c + 1]]
        assert np.all(got[members] == -1)  # each particle in one set only
        got[members] = c
    assert np.array_equal(got, cube)


def test_particle_sets_follow_the_particles():
    spec = moving_box()
    parts = W.surface_particles(spec, seed=13)
    g = bcm.Grid(spec, bcm.PREC_F64)
    g.load_state(W.initial_state(spec, seed=2, noise=1e-2))
    g.set_particles(parts)
    X0, _, cube0 = g.particles()
    assert np.array_equal(X0, parts.X)
    check_sets(g, spec, X0)
    g.step(3, rtol=1e-12)
    X, _, cube = g.particles()
    assert not np.array_equal(X, X0)
    check_sets(g, spec, X)
    assert np.array_equal(cube, expected_sets(spec, X))


def run_both(spec, parts, prec, steps, state, rtol=1e-13, graph=False):
    o = O.Oracle(spec)
    ost = o.new_state(state)
    Xo = parts.X.copy()
    ostats, rc, Fo = o.step_particles(ost, Xo, parts, nsteps=steps, rtol=1e-13)
    assert rc == 0
    g = bcm.Grid(spec, prec)
    g.load_state(state)
    g.set_particles(parts)
    st = (g.step_graph if graph else g.step)(steps, rtol=rtol if prec == bcm.PREC_F64 else 1e-12)
    X, F, _ = g.particles()
    return g, st, X, F, ost, ostats, Xo, Fo


def velocity(g):
    return np.concatenate([g.numpy(f) for f in (bcm.U, bcm.V, bcm.W)])


@pytest.mark.parametrize("prec", [bcm.PREC_F64, bcm.PREC_F32_REFINE])
@pytest.mark.parametrize("name", ["sphere_B8", "moving_box"])
def test_particle_steps_match_oracle(name, prec):
    spec = GRIDS[name]()
    parts = W.surface_particles(spec, seed=21)
    state = W.initial_state(spec, seed=22, noise=1e-3)
    if name == "moving_box":  # a uniform stream through the box
        state.u[:] += 0.3
    g, st, X, F, ost, ostats, Xo, Fo = run_both(spec, parts, prec, 3, state)
    tol = TOL64 if prec == bcm.PREC_F64 else TOL32
    ref = np.concatenate([ost[k] for k in "uvw"])
    assert rel_l2(velocity(g), ref) <= tol
    assert rel_l2(demean_per_sim(g.numpy(bcm.P), spec), demean_per_sim(ost["p"], spec)) <= tol
    assert np.abs(X - Xo).max() <= 1e-13
    assert rel_l2(F, Fo) <= (1e-9 if prec == bcm.PREC_F64 else 1e-4)
    assert rel_l2(st[0]["drag"], ostats[0]["drag"]) <= (1e-9 if prec == bcm.PREC_F64 else 1e-4)
    assert st[0]["converged"] == 1


def test_batched_sims_with_particles():
    spec = W.concat([sphere(8), W.cavity(2, 8, re=200.0), sphere(8, nx=2, ny=2, nz=2)])
    spec.bodies[2] = [W.Body(W.BODY_SPHERE, np.array([0.5, 0.5, 0.5]), np.array([0.15] * 3),
                             omega=np.array([0.0, 0.0, 1.5]))]
    parts = W.concat_particles([W.surface_particles(spec, sim=0, seed=1),
                                W.surface_particles(spec, sim=2, seed=2)])
    state = W.initial_state(spec, seed=23, noise=1e-3)
    g, st, X, F, ost, ostats, Xo, Fo = run_both(spec, parts, bcm.PREC_F64, 2, state)
    ref = np.concatenate([ost[k] for k in "uvw"])
    assert rel_l2(velocity(g), ref) <= TOL64
    assert np.abs(X - Xo).max() <= 1e-13
    for s in range(3):
        assert np.allclose(st[s]["drag"], ostats[s]["drag"], rtol=1e-9, atol=1e-12)
    assert st[1]["drag"] == [0.0, 0.0, 0.0]


def test_graph_steps_with_particles():
    spec = moving_box()
    parts = W.surface_particles(spec, seed=31)
    state = W.initial_state(spec, seed=32, noise=1e-3)
    state.u[:] += 0.3
    g, st, X, F, ost, ostats, Xo, Fo = run_both(spec, parts, bcm.PREC_F32_REFINE, 3, state,
                                                graph=True)
    ref = np.concatenate([ost[k] for k in "uvw"])
    assert rel_l2(velocity(g), ref) <= TOL32
    assert np.abs(X - Xo).max() <= 1e-13


def test_particles_rejected_where_not_defined():
    two = W.two_level_channel(4, 4, 4, 8, (1, 1, 1), (3, 3, 3), 1 / 16., 0)
    g = bcm.Grid(two, bcm.PREC_F64)
    parts = W.Particles(np.array([[0.5, 0.5, 0.5]]), np.zeros(1, np.int32),
                        np.zeros(1, np.int32), np.ones(1))
    with pytest.raises(bcm.BCMError) as ei:
        g.set_particles(parts)
    assert ei.value.status == bcm.BCM_E_INVALID
    spec = sphere(8)
    g = bcm.Grid(spec, bcm.PREC_F64)
    outside = W.Particles(np.array([[0.5, 0.5, 0.5], [5.0, 0.5, 0.5]]), np.zeros(2, np.int32),
                          np.zeros(2, np.int32), np.ones(2))
    with pytest.raises(bcm.BCMError) as ei:
        g.set_particles(outside)
    assert ei.value.status == bcm.BCM_E_BOUNDS
    bad = W.Particles(np.array([[0.5, 0.5, 0.5]]), np.zeros(1, np.int32),
                      np.full(1, 7, np.int32), np.ones(1))
    with pytest.raises(bcm.BCMError) as ei:
        g.set_particles(bad)
    assert ei.value.status == bcm.BCM_E_INVALID
    # back to the solid fraction: the grid steps as before the particles
    g.set_particles(None)
    g.load_state(W.initial_state(spec, seed=3, noise=1e-3))
    assert g.step(1, rtol=1e-10)[0]["converged"] == 1


def test_full_size_sphere_particles_mixed():
    """The 4.19M-cell sphere flow with its surface particles: two mixed steps against
    two FP64 steps on the GPU (1e-6), drag within 1e-4."""
    spec = W.config_sphere(2)
    parts = W.surface_particles(spec)
    state = W.initial_state(spec)
    out = []
    for prec in (bcm.PREC_F32_REFINE, bcm.PREC_F64):
        g = bcm.Grid(spec, prec)
        g.load_state(state)
        g.set_particles(parts)
        st = g.step(2, rtol=1e-10)
        assert st[0]["converged"] == 1
        out.append((velocity(g), st[0]["drag"]))
        del g
        torch.cuda.empty_cache()
    assert rel_l2(out[0][0], out[1][0]) <= TOL32
    assert rel_l2(out[0][1], out[1][1]) <= 1e-4
    assert out[1][1][0] > 0  # the flow pushes the sphere downstream
