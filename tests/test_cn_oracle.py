"""Pins of the oracle's QUICK + Crank-Nicolson momentum scheme (R20 in oracle/bcm_oracle.c)
to things other than itself: QUICK's conservative flux difference is exact for cubic
profiles carried by a uniform stream and, for a quartic, exceeds the exact face-value
difference by (3/2)|U| h^3 for either sign of U (worked out by hand from the quadratic
upstream interpolation: the upwind direction decides that sign); one Crank-Nicolson
step of a divergence-free shear mode decays by the Crank-Nicolson amplification factor
of the discrete Laplacian eigenvalue; a uniform stream is a fixed point; switching back
to Adams-Bashforth restarts it with the Euler step."""
import numpy as np
import pytest

import oracle as O
from paper_1808_04099_gb300 import workloads as W


def _centres(spec):
    B = spec.B
    h = spec.sim_h0[0]
    i = np.arange(B) + 0.5
    cc = np.asarray(spec.cube_ijk, np.float64).reshape(-1, 1, 1, 1, 3)
    k3, j3, i3 = np.meshgrid(i, i, i, indexing="ij")
    off = np.stack([i3, j3, k3], axis=-1)[None]
    return (spec.sim_origin[0] + h * (cc + off)).reshape(-1, 3)


def _channel():
    return W.sphere_channel(4, 2, 2, 8, length=(2.0, 1.0, 1.0), radius=0.2)


def _interior(spec, x, m=2):
    h = spec.sim_h0[0]
    L = spec.sim_extent[0] * h
    return np.all((x > m * h) & (x < L - m * h), axis=1)


@pytest.mark.parametrize("U0", [0.7, -0.4])
def test_quick_is_exact_for_cubics(U0):
    spec = _channel()
    o = O.Oracle(spec)
    x = _centres(spec)
    a, b, c, d = 0.3, -0.8, 0.5, 0.9
    v = a + b * x[:, 0] + c * x[:, 0] ** 2 + d * x[:, 0] ** 3
    u = np.full(spec.n_cells, U0)
    ub = W.initial_state(spec).ub
    N = o.convection_quick(u, v, np.zeros(spec.n_cells), ub)[1]
    inner = _interior(spec, x)
    exact = U0 * (b + 2 * c * x[:, 0] + 3 * d * x[:, 0] ** 2 + d * spec.sim_h0[0] ** 2 / 4)
    assert np.abs(N[inner] - exact[inner]).max() <= 1e-11 * np.abs(exact).max()


@pytest.mark.parametrize("U0", [0.7, -0.4])
def test_quick_quartic_error_is_upwind_dissipative(U0):
    spec = _channel()
    o = O.Oracle(spec)
    x = _centres(spec)
    h = spec.sim_h0[0]
    v = x[:, 0] ** 4
    ub = W.initial_state(spec).ub
    N = o.convection_quick(np.full(spec.n_cells, U0), v, np.zeros(spec.n_cells), ub)[1]
    inner = _interior(spec, x)
    face_diff = ((x[:, 0] + h / 2) ** 4 - (x[:, 0] - h / 2) ** 4) / h
    want = U0 * face_diff + 1.5 * abs(U0) * h ** 3
    assert np.abs(N[inner] - want[inner]).max() <= 1e-11 * np.abs(want).max()


def _shear_box(nu=0.05):
    spec = W.periodic_box(2, 8, nu=nu)
    spec.bodies[0] = []
    return spec


def test_crank_nicolson_decays_a_shear_mode_by_its_amplification_factor():
    """u = A sin(y): divergence free, its convection vanishes discretely, and the
    7-point Laplacian has the eigenvalue lambda = (2 - 2 cos h) / h^2 on it; one
    Crank-Nicolson step multiplies it by (1 - dt nu lambda / 2) / (1 + dt nu lambda / 2)."""
    spec = _shear_box()
    o = O.Oracle(spec)
    o.set_scheme(1, 1e-14, 500)
    x = _centres(spec)
    A = 0.8
    st = o.new_state(W.initial_state(spec))
    st["u"][:] = A * np.sin(x[:, 1])
    st["v"][:] = 0.0
    st["w"][:] = 0.0
    st["p"][:] = 0.0
    stats, rc = o.step(st, 1, rtol=1e-13)
    assert rc == 0
    h, dt, nu = spec.sim_h0[0], spec.sim_dt[0], spec.sim_nu[0]
    lam = (2 - 2 * np.cos(h)) / h ** 2
    R = (1 - 0.5 * dt * nu * lam) / (1 + 0.5 * dt * nu * lam)
    assert np.abs(st["u"] - R * A * np.sin(x[:, 1])).max() <= 1e-12
    assert np.abs(st["v"]).max() <= 1e-14 and np.abs(st["w"]).max() <= 1e-14
    # the explicit Euler factor differs by (dt nu lambda)^2 / 2, far above the pin's
    # tolerance: the pin separates the schemes
    assert abs(R - (1 - dt * nu * lam)) * A > 1e6 * 1e-12


def test_uniform_stream_is_a_fixed_point():
    spec = _shear_box()
    o = O.Oracle(spec)
    o.set_scheme(1, 1e-14, 500)
    st = o.new_state(W.initial_state(spec))
    U = (0.3, -0.2, 0.45)
    for e, k in enumerate("uvw"):
        st[k][:] = U[e]
    st["p"][:] = 0.0
    stats, rc = o.step(st, 2, rtol=1e-13)
    assert rc == 0
    for e, k in enumerate("uvw"):
        assert np.abs(st[k] - U[e]).max() <= 1e-14


def test_switching_back_restarts_adams_bashforth():
    """Steps with Crank-Nicolson, then Adams-Bashforth again: the first AB2 step after
    the switch equals an Euler-started step from the same state (N^{n-1} := N^n)."""
    spec = W.sphere_channel(4, 2, 2, 8, radius=0.3)
    st0 = W.initial_state(spec, seed=4, noise=1e-3)
    o = O.Oracle(spec)
    a = o.new_state(st0)
    o.set_scheme(1, 1e-12, 200)
    o.step(a, 1, rtol=1e-12)
    o.set_scheme(0)
    snap = {k: v.copy() for k, v in a.items()}
    o.step(a, 1, rtol=1e-12)
    o2 = O.Oracle(spec)
    b = {k: v.copy() for k, v in snap.items()}
    b["step"][:] = 0  # an Euler start, at the same body time (the sphere is fixed)
    o2.step(b, 1, rtol=1e-12)
    for k in "uvwp":
        assert np.array_equal(a[k], b[k]), k


AFFINE_GRIDS = {
    "cavity_walls_and_lid": lambda: W.cavity(2, 4),
    "channel_inflow_modes_outflow_slip": lambda: W.sphere_channel(
        2, 1, 1, 4, length=(2.0, 1.0, 1.0), modes=[0.1, -0.05, 0.02, 0.0, 0.03, 0.0, 0.0, 0.01]),
    "periodic": lambda: W.periodic_box(2, 4),
    "two_level_21_faces": lambda: W.two_level_channel(4, 4, 4, 4, (1, 1, 1), (3, 3, 3), 1 / 8., 0),
}


@pytest.mark.parametrize("name", sorted(AFFINE_GRIDS))
def test_velocity_ghosts_are_affine(name):
    """The velocity halo rules are affine in the field once the boundary values are
    fixed: the ghosts of u + d minus the ghosts of u are the same for every u.  This
    holds for same-level copies, 2:1 injection and means, walls, inflow with modes,
    slip and convective outflow with given face values.  It is what lets an iteration
    on the increment d take the neighbour sum of d from the tiles of u^n + d, with the
    sum over u^n folded once into the explicit term."""
    spec = AFFINE_GRIDS[name]()
    o = O.Oracle(spec)
    rng = np.random.default_rng(81)
    ns = len(W.outflow_slots(spec))
    ub = rng.standard_normal((ns, 3, spec.B, spec.B)) if ns else None
    for kind in range(3):
        u1, u2, d = rng.standard_normal((3, spec.n_cells))
        a = o.fill_ghosts(u1 + d, kind, ub) - o.fill_ghosts(u1, kind, ub)
        b = o.fill_ghosts(u2 + d, kind, ub) - o.fill_ghosts(u2, kind, ub)
        assert np.abs(a).max() > 0.1  # the ghosts of d are not all zero
        assert np.allclose(a, b, rtol=0, atol=1e-13), (kind, np.abs(a - b).max())
