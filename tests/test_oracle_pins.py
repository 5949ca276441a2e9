"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a monolithic
array (halo copies), closed forms (quadratics, linear fields, Taylor-Green decay),
invariants (symmetry, null space, divergence after projection), a dense direct
solve on tiny grids, or brute force.  Paper passages: "Building Cube Method"
(halo, cell centres), "Numerical algorithm" (Eq. substep1, Eq. poisson).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1808_04099_gb300 import workloads as W


def cube_view(f, spec):
    B = spec.B
    return np.asarray(f).reshape(spec.n_cubes, B, B, B)  # [c, k, j, i]


def monolithic(f, spec):
    """Assemble a single-level, single-sim cube field into one [z, y, x] array."""
    B = spec.B
    ext = spec.sim_extent[0]
    out = np.full((ext[2], ext[1], ext[0]), np.nan)
    fv = cube_view(f, spec)
    for c in range(spec.n_cubes):
        x, y, z = spec.cube_ijk[c]
        out[z:z + B, y:y + B, x:x + B] = fv[c]
    return out


def centres(spec):
    """Cell-centre coordinates (Eq. cell-center) of every cell, cube-major."""
    B = spec.B
    hf = spec.sim_h0[0] / 2 ** spec.max_level
    X = np.zeros((spec.n_cubes, B, B, B, 3))
    ar = np.arange(B) + 0.5
    for c in range(spec.n_cubes):
        h = spec.sim_h0[0] / 2 ** int(spec.cube_level[c])
        base = spec.sim_origin[0] + spec.cube_ijk[c] * hf
        X[c, ..., 0] = base[0] + ar[None, None, :] * h
        X[c, ..., 1] = base[1] + ar[None, :, None] * h
        X[c, ..., 2] = base[2] + ar[:, None, None] * h
    return X.reshape(-1, 3)


# ----------------------------------------------------------------- adjacency

def test_neighbors_periodic_brute_force():
    spec = W.periodic_box(3, 4)
    nb = O.Oracle(spec).neighbors()
    pos = {tuple(p): c for c, p in enumerate(spec.cube_ijk // 4)}
    for c, p in enumerate(spec.cube_ijk // 4):
        for f in range(6):
            d, side = f // 2, f % 2
            q = list(p)
            q[d] = (q[d] + (1 if side else -1)) % 3
            assert nb[c, f] == pos[tuple(q)]


def test_neighbors_walls_and_slots():
    spec = W.sphere_channel(4, 2, 2, 4)
    o = O.Oracle(spec)
    nb = o.neighbors()
    assert o.n_slots == len(W.outflow_slots(spec)) == 4
    for c, p in enumerate(spec.cube_ijk // 4):
        for f in range(6):
            d, side = f // 2, f % 2
            edge = (p[d] == (spec.sim_extent[0][d] // 4 - 1)) if side else (p[d] == 0)
            assert (nb[c, f] == -1) == edge


# ----------------------------------------------------------------------- halo

def test_halo_equals_monolithic_periodic():
    """Same-level halo copy: ghosts equal the neighbouring cells of one big array."""
    spec = W.periodic_box(3, 4)
    rng = np.random.default_rng(1)
    f = rng.standard_normal(spec.n_cells)
    g = O.Oracle(spec).fill_ghosts(f, 3)
    M = monolithic(f, spec)
    n = M.shape[0]
    B, H = 4, 2
    for c in range(spec.n_cubes):
        x, y, z = spec.cube_ijk[c]
        for axis in range(3):
            for layer in range(1, H + 1):
                for side in (-1, 1):
                    idx = [slice(H, H + B)] * 3   # ghosted buffer [k, j, i]
                    gl = [np.arange(z, z + B), np.arange(y, y + B), np.arange(x, x + B)]
                    ax = 2 - axis
                    pos = (H - layer) if side < 0 else (H + B - 1 + layer)
                    idx[ax] = pos
                    start = (z, y, x)[ax]
                    gl[ax] = np.array([(start - layer) % n if side < 0 else (start + B - 1 + layer) % n])
                    want = M[np.ix_(gl[0], gl[1], gl[2])].squeeze(axis=ax)
                    assert np.array_equal(g[c][tuple(idx)], want)


def test_halo_boundary_face_values():
    """Wall/inflow ghosts put the face value (mean of ghost and interior) at the
    prescribed velocity; slip makes the normal face value zero and the tangential
    gradient zero; outflow pressure ghosts make the face value zero."""
    spec = W.cavity(2, 4)
    o = O.Oracle(spec)
    rng = np.random.default_rng(2)
    B, H = 4, 2
    for kind in range(3):
        f = rng.standard_normal(spec.n_cells)
        g = o.fill_ghosts(f, kind)
        fv = cube_view(f, spec)
        for c in range(spec.n_cubes):
            if spec.cube_ijk[c][2] == 4:  # top layer of cubes: +z is the lid
                face = 0.5 * (g[c][H + B, H:H + B, H:H + B] + fv[c][B - 1])
                assert np.allclose(face, [1.0, 0, 0][kind], atol=1e-15, rtol=0)
    spec = W.sphere_channel(2, 1, 1, 4, length=(2.0, 1.0, 1.0), center=(9, 9, 9))
    o = O.Oracle(spec)
    for kind in range(4):
        f = rng.standard_normal(spec.n_cells)
        g = o.fill_ghosts(f, kind, np.zeros((1, 3, B, B)))
        fv = cube_view(f, spec)
        lower_y = g[0][H:H + B, H - 1, H:H + B]
        if kind == 1:
            assert np.array_equal(lower_y + fv[0][:, 0, :], np.zeros((B, B)))
        else:
            assert np.array_equal(lower_y, fv[0][:, 0, :])
        if kind == 3:  # pressure: Dirichlet 0 at the outflow (+x of cube 1)
            assert np.array_equal(g[1][H:H + B, H:H + B, H + B] + fv[1][:, :, B - 1],
                                  np.zeros((B, B)))


def test_halo_two_level_linear_field():
    """Fine->coarse ghost = mean of 8 fine cells, exact at the coarse ghost centre for a
    linear field; coarse->fine ghost = the covering coarse cell's value (injection)."""
    spec = W.two_level_channel(4, 2, 2, 4, (1, 0, 0), (3, 2, 2), 1 / 8., 0)
    o = O.Oracle(spec)
    X = centres(spec)
    a = np.array([0.3, -1.1, 0.7])
    f = X @ a + 0.25
    g = o.fill_ghosts(f, 3)
    nb = o.neighbors()
    B, H = 4, 2
    hf = spec.sim_h0[0] / 2
    checked = [0, 0]
    for c in range(spec.n_cubes):
        lev = int(spec.cube_level[c])
        h = spec.sim_h0[0] / 2 ** lev
        base = spec.cube_ijk[c] * hf
        for fc in range(6):
            d, side = fc // 2, fc % 2
            if nb[c, fc] not in (-2, -3):
                continue
            # ghost layer 1 along d, all tangential cells
            for t1 in range(B):
                for t2 in range(B):
                    ijk = [0, 0, 0]
                    ijk[d] = -1 if side == 0 else B
                    others = [e for e in range(3) if e != d]
                    ijk[others[0]], ijk[others[1]] = t1, t2
                    val = g[c][ijk[2] + H, ijk[1] + H, ijk[0] + H]
                    xg = base + (np.array(ijk) + 0.5) * h
                    if nb[c, fc] == -3:       # coarse cube, fine neighbours: exact mean
                        assert abs(val - (xg @ a + 0.25)) < 1e-13
                        checked[0] += 1
                    else:                     # fine cube: value of the coarse cell covering xg
                        hc = 2 * h
                        xc = (np.floor(xg / hc) + 0.5) * hc
                        assert abs(val - (xc @ a + 0.25)) < 1e-13
                        checked[1] += 1
    assert checked[0] > 0 and checked[1] > 0


# ------------------------------------------------------------ pressure operator

@pytest.mark.parametrize("spec", [
    W.cavity(2, 4), W.sphere_channel(4, 2, 2, 4),
    W.two_level_channel(4, 2, 2, 4, (1, 0, 0), (3, 2, 2), 1 / 8., 0), W.periodic_box(2, 4)],
    ids=["cavity", "channel", "two_level", "periodic"])
def test_poisson_operator_symmetric_psd(spec):
    o = O.Oracle(spec)
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal((2, spec.n_cells))
    Kx, Ky = o.apply_poisson(x), o.apply_poisson(y)
    assert abs(x @ Ky - Kx @ y) <= 1e-13 * np.linalg.norm(Kx) * np.linalg.norm(y)
    assert x @ Kx > 0.0
    d = o.poisson_diag()
    # the diagonal is K applied to unit vectors, sampled
    for q in rng.integers(0, spec.n_cells, 8):
        e = np.zeros(spec.n_cells)
        e[q] = 1.0
        assert abs(o.apply_poisson(e)[q] - d[q]) < 1e-15


def test_poisson_null_space_neumann():
    spec = W.cavity(2, 4)
    y = O.Oracle(spec).apply_poisson(np.ones(spec.n_cells))
    assert np.array_equal(y, np.zeros_like(y))


def test_poisson_quadratic_exact():
    """K = -V * Laplacian: on p = x^2 - 0.5 y^2 + 2 z^2 the interior value is -V*(2 - 1 + 4)."""
    spec = W.cavity(3, 4)
    X = centres(spec)
    p = X[:, 0] ** 2 - 0.5 * X[:, 1] ** 2 + 2 * X[:, 2] ** 2
    Kp = O.Oracle(spec).apply_poisson(p)
    h = spec.sim_h0[0]
    interior = np.all((X > 1.5 * h) & (X < 1 - 1.5 * h), axis=1)
    assert interior.sum() > 100
    assert np.allclose(Kp[interior], -h ** 3 * 5.0, rtol=1e-10, atol=0)


def dense_K(o, n):
    K = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        K[:, q] = o.apply_poisson(e)
    return K


def test_pcg_matches_dense_solve_dirichlet():
    spec = W.sphere_channel(2, 2, 2, 4, length=(1.0, 1.0, 1.0), center=(9, 9, 9))
    o = O.Oracle(spec)
    n = spec.n_cells
    rng = np.random.default_rng(4)
    b = rng.standard_normal(n)
    p, st, rc = o.solve_pressure(b, rtol=1e-13)
    assert rc == 0
    V = spec.sim_h0[0] ** 3
    ref = np.linalg.solve(dense_K(o, n), -V * b)
    assert np.linalg.norm(p - ref) <= 1e-11 * np.linalg.norm(ref)


def test_pcg_matches_dense_solve_two_level():
    spec = W.two_level_channel(2, 1, 1, 4, (1, 0, 0), (2, 1, 1), 1 / 8., 0)
    spec.bodies = [[]]
    o = O.Oracle(spec)
    n = spec.n_cells
    rng = np.random.default_rng(5)
    b = rng.standard_normal(n)
    p, st, rc = o.solve_pressure(b, rtol=1e-13)
    lev = np.repeat(spec.cube_level.astype(int), spec.B ** 3)
    V = (spec.sim_h0[0] / 2.0 ** lev) ** 3
    ref = np.linalg.solve(dense_K(o, n), -V * b)
    assert rc == 0 and np.linalg.norm(p - ref) <= 1e-11 * np.linalg.norm(ref)


def test_pcg_matches_lstsq_neumann():
    spec = W.cavity(2, 4)
    o = O.Oracle(spec)
    n = spec.n_cells
    rng = np.random.default_rng(6)
    b = rng.standard_normal(n)
    p, st, rc = o.solve_pressure(b, rtol=1e-13)
    V = spec.sim_h0[0] ** 3
    ref = np.linalg.lstsq(dense_K(o, n), -V * (b - b.mean()), rcond=None)[0]
    assert rc == 0
    assert np.linalg.norm((p - p.mean()) - (ref - ref.mean())) <= 1e-11 * np.linalg.norm(ref)


def test_pcg_zero_rhs_gives_zero():
    spec = W.sphere_channel(2, 1, 1, 4, length=(2.0, 1.0, 1.0), center=(9, 9, 9))
    p, st, rc = O.Oracle(spec).solve_pressure(np.zeros(spec.n_cells), np.ones(spec.n_cells))
    assert rc == 0 and st[0]["cg_iters"] == 0 and not p.any()


# ---------------------------------------------------------- momentum operators

def tg_fields(X):
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = np.cos(x) * np.sin(y) * np.cos(z) * 0.5
    w = np.cos(x) * np.cos(y) * np.sin(z) * -0.25
    return u, v, w


def tg_exact(X):
    """Closed-form div(u u) and Laplacian of the fields in tg_fields."""
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    s, c = np.sin, np.cos
    u = s(x) * c(y) * c(z)
    v = 0.5 * c(x) * s(y) * c(z)
    w = -0.25 * c(x) * c(y) * s(z)
    ux, uy, uz = c(x) * c(y) * c(z), -s(x) * s(y) * c(z), -s(x) * c(y) * s(z)
    vx, vy, vz = -0.5 * s(x) * s(y) * c(z), 0.5 * c(x) * c(y) * c(z), -0.5 * c(x) * s(y) * s(z)
    wx, wy, wz = 0.25 * s(x) * c(y) * s(z), 0.25 * c(x) * s(y) * s(z), -0.25 * c(x) * c(y) * c(z)
    div = ux + vy + wz
    N = [u * ux + v * uy + w * uz + u * div, u * vx + v * vy + w * vz + v * div,
         u * wx + v * wy + w * wz + w * div]
    L = [-3 * u, -3 * v, -3 * w]
    return N, L


def test_convection_diffusion_second_order():
    errs = []
    for m in (4, 8):
        spec = W.periodic_box(m, 8)
        X = centres(spec)
        u, v, w = tg_fields(X)
        N, L = O.Oracle(spec).convection_diffusion(u, v, w)
        Ne, Le = tg_exact(X)
        errs.append((max(np.abs(N[q] - Ne[q]).max() for q in range(3)),
                     max(np.abs(L[q] - Le[q]).max() for q in range(3))))
    for a, b in zip(errs[0], errs[1]):
        assert 3.7 < a / b < 4.3


def test_convection_diffusion_uniform_flow_zero():
    spec = W.periodic_box(2, 4)
    n = spec.n_cells
    N, L = O.Oracle(spec).convection_diffusion(np.full(n, 0.7), np.full(n, -0.2), np.full(n, 0.1))
    for q in range(3):
        assert not N[q].any() and not L[q].any()


def test_rhs_linear_fields():
    """Face averages are exact for linear fields: div(x, -y, 0) = 0, div(x, 0, 0) = 1."""
    spec = W.periodic_box(2, 4)
    o = O.Oracle(spec)
    X = centres(spec)
    h = spec.sim_h0[0]
    inner = np.all((X > 1.5 * h) & (X < 2 * math.pi - 1.5 * h), axis=1)
    dt = spec.sim_dt[0]
    b = o.rhs(X[:, 0], -X[:, 1], np.zeros(spec.n_cells))
    assert np.allclose(b[inner], 0.0, atol=1e-11)
    b = o.rhs(X[:, 0], np.zeros(spec.n_cells), np.zeros(spec.n_cells))
    assert np.allclose(b[inner] * dt, 1.0, rtol=1e-12)


# ----------------------------------------------------------------- bodies / IB

def test_solid_fraction_sphere_values():
    spec = W.sphere_channel(2, 1, 1, 4, length=(2.0, 1.0, 1.0), radius=0.3, center=(0.5, 0.5, 0.5))
    o = O.Oracle(spec)
    X = centres(spec)
    phi, us, vs, ws = o.solid_fraction(0.0)
    d = np.linalg.norm(X - 0.5, axis=1) - 0.3
    eps = 1.5 * spec.sim_h0[0]
    far = d >= 20 * eps
    assert not phi[far].any()
    # phi decreases with the distance and is 1/2 on the surface
    order = np.argsort(d[~far])
    assert np.all(np.diff(phi[~far][order]) <= 1e-15)
    assert np.allclose(phi[~far], 0.5 * (1 - np.tanh(d[~far] / eps)), rtol=1e-14, atol=1e-16)
    assert not us.any() and not vs.any() and not ws.any()


def test_solid_fraction_ellipsoid_special_cases():
    """Equal semi-axes reduce the ellipsoid estimate to the sphere's exact distance;
    a quarter turn about z swaps the x and y semi-axes."""
    base = W.sphere_channel(2, 1, 1, 4, length=(2.0, 1.0, 1.0), radius=0.3, center=(0.6, 0.5, 0.5))
    o = O.Oracle(base)
    phi_s = o.solid_fraction(0.0)[0]
    e = W.sphere_channel(2, 1, 1, 4, length=(2.0, 1.0, 1.0), radius=0.3, center=(0.6, 0.5, 0.5))
    e.bodies = [[W.Body(W.BODY_ELLIPSOID, np.array([0.6, 0.5, 0.5]), np.array([0.3, 0.3, 0.3]))]]
    assert np.allclose(O.Oracle(e).solid_fraction(0.0)[0], phi_s, rtol=1e-12, atol=1e-15)
    a = np.array([0.35, 0.2, 0.25])
    e.bodies = [[W.Body(W.BODY_ELLIPSOID, np.array([0.6, 0.5, 0.5]), a)]]
    phi_a = O.Oracle(e).solid_fraction(0.0)[0]
    q = np.array([math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)])
    e.bodies = [[W.Body(W.BODY_ELLIPSOID, np.array([0.6, 0.5, 0.5]), a[[1, 0, 2]], q)]]
    assert np.allclose(O.Oracle(e).solid_fraction(0.0)[0], phi_a, rtol=1e-12, atol=1e-15)
    # the same quarter turn reached by rotating for a time t about z from identity
    om = np.array([0, 0, 0.5])
    e.bodies = [[W.Body(W.BODY_ELLIPSOID, np.array([0.6, 0.5, 0.5]), a[[1, 0, 2]],
                        np.array([1.0, 0, 0, 0]), om)]]
    phi_t, us, vs, ws = O.Oracle(e).solid_fraction(math.pi)
    assert np.allclose(phi_t, phi_a, rtol=1e-12, atol=1e-15)
    X = centres(e)
    near = phi_t > 0
    assert np.allclose(us[near], -0.5 * (X[near, 1] - 0.5), atol=1e-14)
    assert np.allclose(vs[near], 0.5 * (X[near, 0] - 0.6), atol=1e-14)


# ------------------------------------------------------------------- the step

def test_projection_divergence_equals_residual():
    for spec in (W.cavity(2, 4), W.sphere_channel(4, 2, 2, 4)):
        o = O.Oracle(spec)
        st = o.new_state(W.initial_state(spec, 0, 1e-3))
        stats, rc = o.step(st, 2, rtol=1e-11)
        assert rc == 0
        s = stats[0]
        assert s["rel_resid"] <= 1e-11 and s["div_rel"] <= 1.5e-11
        assert abs(s["div_rel"] - s["rel_resid"]) <= 1e-3 * s["rel_resid"] + 1e-15


def test_uniform_flow_fixed_point():
    spec = W.sphere_channel(4, 2, 2, 4, center=(90, 90, 90))
    o = O.Oracle(spec)
    st = o.new_state(W.initial_state(spec))
    stats, rc = o.step(st, 3)
    assert np.abs(st["u"] - 1).max() < 1e-14
    assert np.abs(st["v"]).max() < 1e-14 and np.abs(st["w"]).max() < 1e-14
    assert np.abs(st["p"]).max() < 1e-14


def test_far_body_is_bitwise_no_body():
    a = W.sphere_channel(4, 2, 2, 4, center=(90, 90, 90))
    b = W.sphere_channel(4, 2, 2, 4, center=(90, 90, 90))
    b.bodies = [[]]
    res = []
    for spec in (a, b):
        o = O.Oracle(spec)
        st = o.new_state(W.initial_state(spec, 3, 1e-2))
        o.step(st, 2)
        res.append(st)
    for k in ("u", "v", "w", "p"):
        assert np.array_equal(res[0][k], res[1][k])


def test_body_covering_periodic_box_imposes_its_velocity():
    spec = W.periodic_box(2, 4)
    spec.bodies = [[W.Body(W.BODY_SPHERE, np.array([3.0, 3.0, 3.0]), np.array([100.0] * 3),
                           vel=np.array([0.3, -0.1, 0.2]))]]
    o = O.Oracle(spec)
    st = o.new_state(W.initial_state(spec, 4, 0.5))
    o.step(st, 1)
    # phi == 1 everywhere: u* = u~ + (u_s - u~) = u_s up to one rounding, then the
    # projection of a uniform field leaves it unchanged
    assert np.abs(st["u"] - 0.3).max() < 1e-14
    assert np.abs(st["v"] + 0.1).max() < 1e-14
    assert np.abs(st["w"] - 0.2).max() < 1e-14


def test_drag_points_downstream():
    spec = W.sphere_channel(4, 2, 2, 8)
    o = O.Oracle(spec)
    st = o.new_state(W.initial_state(spec))
    stats, rc = o.step(st, 2)
    dx, dy, dz = stats[0]["drag"]
    assert dx > 0 and abs(dy) < 1e-6 * dx and abs(dz) < 1e-6 * dx


def taylor_green_error(m, B=8, nu=0.05, T=0.3):
    """2-D Taylor-Green vortex u = sin x cos y e^{-2 nu t}, v = -cos x sin y e^{-2 nu t}."""
    spec = W.periodic_box(m, B, nu)
    h = spec.sim_h0[0]
    nsteps = int(math.ceil(T / (0.2 * h)))
    spec.sim_dt[:] = T / nsteps
    o = O.Oracle(spec)
    X = centres(spec)
    st0 = W.initial_state(spec)
    st0.u = np.sin(X[:, 0]) * np.cos(X[:, 1])
    st0.v = -np.cos(X[:, 0]) * np.sin(X[:, 1])
    st = o.new_state(st0)
    ke = [0.5 * (st["u"] ** 2 + st["v"] ** 2).sum()]
    for _ in range(nsteps):
        o.step(st, 1, rtol=1e-12)
        ke.append(0.5 * (st["u"] ** 2 + st["v"] ** 2 + st["w"] ** 2).sum())
    decay = math.exp(-2 * nu * T)
    ue = np.sin(X[:, 0]) * np.cos(X[:, 1]) * decay
    err = np.linalg.norm(st["u"] - ue) / np.linalg.norm(ue)
    return err, np.array(ke), np.abs(st["w"]).max()


def test_taylor_green_decay_converges():
    e1, ke1, w1 = taylor_green_error(2)
    e2, ke2, w2 = taylor_green_error(4)
    assert e2 < e1 / 3.0 and e2 < 5e-3
    assert np.all(np.diff(ke2) < 0)             # kinetic energy decays monotonically
    assert w2 < 1e-12                            # stays two-dimensional


# ------------------------------------------------ Adams-Bashforth combination (R3)

def test_ab2_transverse_mode_follows_the_recurrence():
    """A uniform stream u = U carrying a transverse mode v = eps sin(k x) through the
    all-periodic box.  With u uniform and v constant along y and z, the conservative
    central convection of v is exactly U times the central difference of v, that of u
    and w is zero, the Laplacian acts on the mode by its discrete eigenvalue, and every
    face divergence is zero, so the pressure stays zero and the projection leaves the
    field alone.  The complex amplitude a of v = Re(a e^{ikx}) then follows the
    Adams-Bashforth-2 recurrence of the momentum sub-step (Euler first step, R3):
        a_1     = a_0 + dt (-s a_0 - nu lam a_0)
        a_{n+1} = a_n + dt (-(3/2 s a_n - 1/2 s a_{n-1}) - nu lam a_n)
    with s = i U sin(kh)/h and lam = (4/h^2) sin^2(kh/2).  A wrong weight, sign or lag
    in the combination (or Euler throughout) is off by O(dt^2 |s|^2 |a|) per step, far
    above the 1e-12 held here."""
    spec = W.periodic_box(2, 8, nu=0.05)
    h, dt, nu = spec.sim_h0[0], spec.sim_dt[0], spec.sim_nu[0]
    U, eps, k = 1.0, 0.1, 2.0
    X = centres(spec)
    st0 = W.initial_state(spec)
    st0.u = np.full(spec.n_cells, U)
    st0.v = eps * np.sin(k * X[:, 0])
    st0.w = np.zeros(spec.n_cells)
    o = O.Oracle(spec)
    st = o.new_state(st0)
    s = 1j * U * math.sin(k * h) / h
    lam = 4.0 / h ** 2 * math.sin(k * h / 2) ** 2
    a_prev, a = None, -1j * eps
    phase = np.exp(1j * k * X[:, 0])
    for n in range(4):
        stats, rc = o.step(st, 1, rtol=1e-13)
        assert rc == 0
        if n == 0:
            a_next = a + dt * (-s * a - nu * lam * a)
        else:
            a_next = a + dt * (-(1.5 * s * a - 0.5 * s * a_prev) - nu * lam * a)
        a_prev, a = a, a_next
        v_exact = np.real(a * phase)
        assert np.abs(st["v"] - v_exact).max() <= 1e-12 * eps, n
        assert np.abs(st["u"] - U).max() <= 1e-13 and np.abs(st["w"]).max() <= 1e-13
        assert np.abs(st["p"]).max() <= 1e-12
    # the recurrence is not the Euler one: after four steps the two differ clearly
    a_e = -1j * eps
    for n in range(4):
        a_e = a_e + dt * (-s * a_e - nu * lam * a_e)
    assert abs(a_e - a) > 1e3 * 1e-12 * eps


# ------------------------------------------------ convective outflow face values (R8)

def test_outflow_face_values_advance_by_the_convective_update():
    """Outflow face values away from the interior values: one step advances each face
    value by the explicit convective update of R8, u_b^{n+1} = u_b^n - U_c dt (u_b^n -
    u_0^n) / (h/2), u_0 the interior cell next to the face at t^n (not the face-to-
    centre distance h, and with the sign that relaxes u_b towards u_0)."""
    spec = W.sphere_channel(4, 2, 2, 4, center=(90, 90, 90))
    B = spec.B
    rng = np.random.default_rng(12)
    st0 = W.initial_state(spec, 3, 0.2)
    st0.ub = st0.ub + rng.uniform(-0.3, 0.3, st0.ub.shape)
    o = O.Oracle(spec)
    st = o.new_state(st0)
    stats, rc = o.step(st, 1, rtol=1e-12)
    assert rc == 0
    h, dt, Uc = spec.sim_h0[0], spec.sim_dt[0], spec.sim_uconv[0]
    slots = W.outflow_slots(spec)
    assert len(slots) > 0
    ub1 = st["ub"].reshape(st0.ub.shape)
    vel = [cube_view(f, spec) for f in (st0.u, st0.v, st0.w)]  # [c, k, j, i]
    for sl, (c, f) in enumerate(slots):
        assert f == 1  # +x outflow: tangential a = y (fastest), b = z
        for comp in range(3):
            u0 = vel[comp][c, :, :, B - 1]          # [b = z, a = y]
            ub0 = st0.ub[sl, comp]
            expect = ub0 - Uc * dt * (ub0 - u0) / (0.5 * h)
            assert np.abs(ub1[sl, comp] - expect).max() <= 1e-15 * (1 + np.abs(expect).max())
    # the update moves every face value: u_b^n - u_0^n is nowhere zero here
    assert np.abs(ub1 - st0.ub).min() > 0.0
