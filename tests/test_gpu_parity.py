"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the
same seeded inputs.

Tolerances (relative L2 per field): FP64 path 1e-10 (velocity vector, each velocity
component and pressure), FP32 sweeps inside FP64 defect correction 1e-6 (velocity
vector and pressure: FP32 storage rounds every component to ~6e-8 of |u|, which is
far more than 1e-6 of a component that is itself small, e.g. the cross-flow
components of a cavity).  Both sides solve the pressure Poisson
equation to a tighter residual than the tolerance so that the solver stopping point
does not dominate the comparison (two CG runs stopped at residual t differ by up
to about cond(K) * t).  Halo fills are compared bit for bit.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1808_04099_gb300 import workloads as W
from _util import demean_per_sim, max_rel, oracle_run, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines, skipped there
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1808_04099_gb300 import bcm  # noqa: E402

TOL64 = 1e-10
TOL32 = 1e-6


def gpu_grid(spec, prec=bcm.PREC_F64, state=None, **kw):
    g = bcm.Grid(spec, prec, **kw)
    if state is not None:
        g.load_state(state)
    return g


MAX_FACTOR = 10.0  # per-cell bound: max |a - b| <= MAX_FACTOR * tol * max |b|


def compare_fields(g, st, spec, tol, per_component=True):
    """Relative L2 error of the velocity field (as a vector) and of the pressure
    (mean removed in all-Neumann sims); with per_component also of u, v, w alone.  Next
    to every relative L2 error, the largest cell error against the largest value, held
    to MAX_FACTOR times the tolerance, so that an error confined to an outflow face, a
    2:1 interface or a body shell cannot hide in the norm."""
    vel = np.concatenate([g.numpy(f) for f in (bcm.U, bcm.V, bcm.W)])
    ref = np.concatenate([st[k] for k in ("u", "v", "w")])
    pg, pr = demean_per_sim(g.numpy(bcm.P), spec), demean_per_sim(st["p"], spec)
    out = {"velocity": rel_l2(vel, ref), "p": rel_l2(pg, pr)}
    mx = {"velocity": max_rel(vel, ref), "p": max_rel(pg, pr)}
    if per_component:
        for name, fid in (("u", bcm.U), ("v", bcm.V), ("w", bcm.W)):
            out[name] = rel_l2(g.numpy(fid), st[name])
            mx[name] = max_rel(g.numpy(fid), st[name])
    for k, v in out.items():
        assert v <= tol, (k, v, out)
    for k, v in mx.items():
        assert v <= MAX_FACTOR * tol, ("max", k, v, mx)
    return out


HALO_SPECS = {
    "periodic": lambda: W.periodic_box(3, 4),
    "cavity": lambda: W.cavity(2, 8),
    "channel": lambda: W.sphere_channel(4, 2, 2, 8),
    "two_level": lambda: W.two_level_channel(4, 2, 2, 8, (1, 0, 0), (3, 2, 2), 1 / 16., 0),
    "B16": lambda: W.sphere_channel(2, 1, 1, 16, length=(2.0, 1.0, 1.0)),
    "two_level_3d": lambda: W.two_level_channel(4, 4, 4, 8, (1, 1, 1), (3, 3, 3), 1 / 16., 0),
}


@pytest.mark.parametrize("name", sorted(HALO_SPECS))
def test_halo_fill_bitwise(name):
    spec = HALO_SPECS[name]()
    rng = np.random.default_rng(7)
    g = gpu_grid(spec)
    o = O.Oracle(spec)
    ub = rng.standard_normal(g.field(bcm.UB).numel())
    g.field(bcm.UB).copy_(torch.from_numpy(ub))
    G = spec.B + 4
    for kind, fid in ((0, bcm.U), (1, bcm.V), (2, bcm.W), (3, bcm.P)):
        f = rng.standard_normal(spec.n_cells)
        g.field(fid).copy_(torch.from_numpy(f))
        got = g.fill_halo(fid, kind).cpu().numpy().reshape(spec.n_cubes, G, G, G)
        want = o.fill_ghosts(f, kind, ub.reshape(-1, 3, spec.B, spec.B) if ub.size else None)
        assert np.array_equal(got, want), (name, kind, np.abs(got - want).max())


@pytest.mark.parametrize("name", ["periodic", "cavity", "channel", "B16", "two_level",
                                  "two_level_3d"])
def test_poisson_operator(name):
    spec = HALO_SPECS[name]()
    x = np.random.default_rng(8).standard_normal(spec.n_cells)
    g = gpu_grid(spec)
    y = g.apply_poisson(torch.from_numpy(x)).cpu().numpy()
    assert rel_l2(y, O.Oracle(spec).apply_poisson(x)) < 1e-14


@pytest.mark.parametrize("name", ["cavity", "channel", "B16", "two_level_3d"])
def test_pressure_solve(name):
    spec = HALO_SPECS[name]()
    b = np.random.default_rng(9).standard_normal(spec.n_cells)
    g = gpu_grid(spec)
    g.field(bcm.RHS).copy_(torch.from_numpy(b))
    st = g.solve_pressure(1e-13)
    assert st[0]["converged"] == 1 and st[0]["rel_resid"] <= 1e-13
    p_ref, ost, rc = O.Oracle(spec).solve_pressure(b, rtol=1e-13)
    p = g.numpy(bcm.P)
    assert rel_l2(demean_per_sim(p, spec), demean_per_sim(p_ref, spec)) < 1e-11
    assert abs(st[0]["cg_iters"] - ost[0]["cg_iters"]) <= 2


STEP_CASES = {
    "cavity_B8": (lambda: W.cavity(2, 8), 1e-3, 4),
    "cavity_B16": (lambda: W.cavity(2, 16), 1e-3, 3),
    "sphere_B8": (lambda: W.sphere_channel(4, 2, 2, 8, radius=0.3), 0.0, 4),
    "periodic_B4": (lambda: W.periodic_box(3, 4), 0.3, 3),
}


@pytest.mark.parametrize("name", sorted(STEP_CASES))
def test_step_fp64(name):
    mk, noise, steps = STEP_CASES[name]
    spec = mk()
    state = W.initial_state(spec, seed=11, noise=noise)
    ost, ostats = oracle_run(spec, state, steps, 1e-13)
    g = gpu_grid(spec, bcm.PREC_F64, state)
    gst = g.step(steps, rtol=1e-13)
    compare_fields(g, ost, spec, TOL64)
    s, r = gst[0], ostats[0]
    assert s["steps"] == steps and s["converged"] == 1
    assert abs(s["div_rel"] - r["div_rel"]) <= 1e-12 + 1e-3 * r["div_rel"]
    for e in range(3):
        assert abs(s["drag"][e] - r["drag"][e]) <= 1e-9 * (abs(r["drag"][0]) + 1e-30)
    assert abs(s["umax"] - r["umax"]) <= 1e-7 * r["umax"]


@pytest.mark.parametrize("name", ["cavity_B8", "sphere_B8", "cavity_B16"])
def test_step_mixed(name):
    mk, noise, steps = STEP_CASES[name]
    spec = mk()
    state = W.initial_state(spec, seed=12, noise=noise)
    ost, ostats = oracle_run(spec, state, steps, 1e-13)
    g = gpu_grid(spec, bcm.PREC_F32_REFINE, state)
    gst = g.step(steps, rtol=1e-12)
    assert gst[0]["converged"] == 1 and gst[0]["refine_cycles"] >= 1
    compare_fields(g, ost, spec, TOL32, per_component=False)


def test_batched_ragged_sims():
    """Several sims of different sizes and kinds in one flattened cube list."""
    specs = [W.cavity(2, 8, re=400.0), W.sphere_channel(4, 2, 2, 8, radius=0.3),
             W.cavity(3, 8, re=150.0), W.sphere_channel(2, 1, 1, 8, length=(2.0, 1.0, 1.0),
                                                        radius=0.2, center=(0.6, 0.5, 0.5))]
    spec = W.concat(specs)
    state = W.initial_state(spec, seed=13, noise=1e-3)
    ost, ostats = oracle_run(spec, state, 3, 1e-13)
    g = gpu_grid(spec, bcm.PREC_F64, state)
    gst = g.step(3, rtol=1e-13)
    compare_fields(g, ost, spec, TOL64)
    for s in range(spec.n_sims):
        assert gst[s]["converged"] == 1
        assert abs(gst[s]["cg_iters"] - ostats[s]["cg_iters"]) <= 3


def test_rotating_ellipsoids():
    spec = W.sphere_channel(4, 2, 2, 8)
    rng = np.random.default_rng(3)
    bodies = []
    for k in range(3):
        q = rng.normal(size=4)
        bodies.append(W.Body(W.BODY_ELLIPSOID, np.array([0.7 + 0.6 * k, 1.0, 1.0]),
                             rng.uniform(0.1, 0.25, 3), q / np.linalg.norm(q),
                             rng.normal(size=3), np.array([0.05, 0, 0])))
    spec.bodies = [bodies]
    state = W.initial_state(spec, seed=14)
    ost, ostats = oracle_run(spec, state, 3, 1e-13)
    g = gpu_grid(spec, bcm.PREC_F64, state)
    gst = g.step(3, rtol=1e-13)
    compare_fields(g, ost, spec, TOL64)
    for e in range(3):
        assert abs(gst[0]["drag"][e] - ostats[0]["drag"][e]) <= 1e-8 * abs(ostats[0]["drag"][0])
    phi_o = O.Oracle(spec).solid_fraction([2 * spec.sim_dt[0]])[0]  # phi of the last step start
    assert rel_l2(g.numpy(bcm.PHI), phi_o) < 1e-12


def test_inflow_modes():
    modes = np.array([0.1, -0.05, 0.02, 0.0, 0.03, -0.01, 0.0, 0.04])
    spec = W.sphere_channel(4, 2, 2, 8, modes=modes)
    state = W.initial_state(spec, seed=15)
    ost, _ = oracle_run(spec, state, 2, 1e-13)
    g = gpu_grid(spec, bcm.PREC_F64, state)
    g.step(2, rtol=1e-13)
    compare_fields(g, ost, spec, TOL64)


def test_not_converged_status():
    spec = W.cavity(2, 8)
    g = gpu_grid(spec, bcm.PREC_F64, W.initial_state(spec, 1, 1e-2))
    with pytest.raises(bcm.BCMError) as ei:
        g.step(1, rtol=1e-14, max_iter=3)
    assert ei.value.status == bcm.BCM_E_NOT_CONVERGED
    st = g.step(1, rtol=1e-14, max_iter=3, allow_not_converged=True)
    assert st[0]["cg_iters"] == 3 and st[0]["converged"] == 0


def test_nonfinite_detected():
    spec = W.cavity(2, 8)
    state = W.initial_state(spec, 1, 1e-2)
    state.u[100] = np.nan
    g = gpu_grid(spec, bcm.PREC_F64, state)
    with pytest.raises(bcm.BCMError) as ei:
        g.step(1, rtol=1e-10)
    assert ei.value.status == bcm.BCM_E_NONFINITE


def test_full_size_sphere_fp64_and_mixed_against_oracle():
    """The sphere flow at its full size (16x8x8 cubes of 16^3, 4.19M cells) in the
    launch configuration the benchmark times, both sides solving to rtol 1e-13: one FP64
    step within 1e-10 of the oracle, and two mixed steps (the FP32 sweeps inside FP64
    defect correction) within 1e-6 of the oracle's two steps; the mixed FP64 residual
    meets its rtol and the corrected face velocities are as divergence free as it says."""
    spec = W.config_sphere(2)
    state = W.initial_state(spec)
    o = O.Oracle(spec)
    ost = o.new_state(state)
    ostats1, rc = o.step(ost, 1, rtol=1e-13)
    assert rc == 0
    one = {k: np.array(v, copy=True) for k, v in ost.items()}
    g = gpu_grid(spec, bcm.PREC_F64, state)
    gst = g.step(1, rtol=1e-13)
    compare_fields(g, one, spec, TOL64)
    assert gst[0]["drag"][0] > 0
    assert abs(gst[0]["drag"][0] - ostats1[0]["drag"][0]) <= 1e-10 * ostats1[0]["drag"][0]
    del g
    ostats2, rc = o.step(ost, 1, rtol=1e-13)
    assert rc == 0
    g32 = gpu_grid(spec, bcm.PREC_F32_REFINE, state)
    s32 = g32.step(2, rtol=1e-12)
    assert s32[0]["converged"] == 1 and s32[0]["rel_resid"] <= 1e-12
    assert s32[0]["div_rel"] <= 1e-11
    compare_fields(g32, ost, spec, TOL32, per_component=False)


def test_full_size_sphere_persistent_forms_mixed():
    """The persistent PCG forms at the benchmark's full size (16x8x8 cubes of 16^3):
    two mixed steps at residual 1e-10 with the streaming form (the default), the
    single-reduction form and the shared-memory form (two cubes per block) meet the
    tolerance and agree."""
    spec = W.config_sphere(2)
    state = W.initial_state(spec)
    runs = []
    for persistent in (1, 2, 3):
        g = gpu_grid(spec, bcm.PREC_F32_REFINE, state)
        g.set_launch(1, 1, persistent=persistent)
        st = g.step(2, rtol=1e-10)
        # 1024 cubes fit one co-resident wave of blocks of two 16^3 tiles (152 SMs x 4)
        assert st[0]["pcg_form"] == persistent
        assert st[0]["converged"] == 1 and st[0]["rel_resid"] <= 1e-10
        assert st[0]["div_rel"] <= 1e-9
        runs.append((np.concatenate([g.numpy(f) for f in (bcm.U, bcm.V, bcm.W)]),
                     st[0]["cg_iters"]))
        del g
    for vel, iters in runs[1:]:
        assert rel_l2(vel, runs[0][0]) <= TOL32
        # same iterates in exact arithmetic: iteration counts within a few percent
        assert abs(iters - runs[0][1]) <= 0.1 * runs[0][1]


@pytest.mark.parametrize("prec", [bcm.PREC_F64, bcm.PREC_F32_REFINE])
def test_launch_shapes_agree(prec):
    """Every PCG launch shape gives the oracle's result: the persistent cooperative
    solver (two passes per iteration with the state on chip, or streamed with 1, 2 or
    4 z-slabs per work item, or the single-reduction form), and the two-launch
    iteration with its slab counts per pass.
    Shapes differ only in rounding."""
    spec = W.sphere_channel(2, 1, 1, 16, length=(2.0, 1.0, 1.0), radius=0.2,
                            center=(0.6, 0.5, 0.5))
    state = W.initial_state(spec, seed=21, noise=1e-3)
    ost, ostats = oracle_run(spec, state, 2, 1e-13)
    tol = TOL64 if prec == bcm.PREC_F64 else TOL32
    shapes = [(1, 1, 1), (1, 2, 1), (1, 4, 1), (3, 1, 1), (3, 2, 1), (2, 1, 1), (2, 2, 1),
              (2, 4, 1), (0, 1, 1), (0, 2, 4), (0, 4, 2), (0, 4, 4)]
    for persistent, sa, sb in shapes:
        g = gpu_grid(spec, prec, state)
        g.set_launch(sa, sb, persistent=persistent)
        st = g.step(2, rtol=1e-13 if prec == bcm.PREC_F64 else 1e-12)
        if persistent:  # the form that ran: on chip only for the FP32 one-slab shape
            on_chip = persistent == 3 and sa == 1 and prec == bcm.PREC_F32_REFINE
            assert st[0]["pcg_form"] == (3 if on_chip else {1: 1, 2: 2, 3: 1}[persistent])
        else:
            assert st[0]["pcg_form"] == 0
        compare_fields(g, ost, spec, tol, per_component=(prec == bcm.PREC_F64))
        if prec == bcm.PREC_F64:
            assert abs(st[0]["cg_iters"] - ostats[0]["cg_iters"]) <= 2


def test_persistent_many_sims_and_fallback():
    """Batched sims through the persistent solver, and the two-launch path that
    grids with more sims than the persistent kernel holds fall back to."""
    specs = [W.cavity(2, 8, re=200.0 + 50 * i) for i in range(5)]
    spec = W.concat(specs)
    state = W.initial_state(spec, seed=22, noise=1e-3)
    ost, _ = oracle_run(spec, state, 2, 1e-13)
    for persistent in (1, 2, 3, 0):
        g = gpu_grid(spec, bcm.PREC_F64, state)
        g.set_launch(1, 1, persistent=persistent)
        g.step(2, rtol=1e-13)
        compare_fields(g, ost, spec, TOL64)


def test_mixed_bf16_lagged_convection():
    """Mixed precision with N^{n-1} stored as bfloat16: the lagged fields are bfloat16,
    and after n steps velocity stays within the error that rounding N^{n-1} can cause:
    each step moves u~ by dt/2 times the rounding of N^{n-1} (at most 2^-9 of |N|,
    bounded here by 2^-8), and the projection does not enlarge it in L2."""
    spec = W.sphere_channel(4, 2, 2, 8, radius=0.3)
    state = W.initial_state(spec, seed=31, noise=1e-3)
    nsteps = 3
    ost, _ = oracle_run(spec, state, nsteps, 1e-13)
    g = gpu_grid(spec, bcm.PREC_F32_REFINE, state, lagged_bf16=True)
    st = g.step(nsteps, rtol=1e-12)
    assert st[0]["converged"] == 1
    assert g.field(bcm.NX).dtype == torch.bfloat16
    vel = np.concatenate([g.numpy(f) for f in (bcm.U, bcm.V, bcm.W)])
    ref = np.concatenate([ost[k] for k in ("u", "v", "w")])
    n_ref = np.concatenate([ost[k] for k in ("nx", "ny", "nz")])
    dt = spec.sim_dt[0]
    bound = nsteps * 0.5 * dt * 2.0 ** -8 * np.linalg.norm(n_ref) / np.linalg.norm(ref) + TOL32
    err = rel_l2(vel, ref)
    assert err <= bound
    # the option is in effect: the result differs from the FP32-stored run
    g32 = gpu_grid(spec, bcm.PREC_F32_REFINE, state)
    g32.step(nsteps, rtol=1e-12)
    vel32 = np.concatenate([g32.numpy(f) for f in (bcm.U, bcm.V, bcm.W)])
    assert rel_l2(vel, vel32) > 0.0


@pytest.mark.parametrize("persistent", [1, 2, 3])
def test_barrier_timeout_reported_and_recovered(persistent):
    """A grid-barrier wait that runs out (a 1 ns limit) ends the persistent solve with
    BCM_E_TIMEOUT instead of waiting; the next solve with the normal limit is exact.
    64 cubes of 16^3: blocks wait microseconds at a barrier, many ticks of the device
    timer, so the 1 ns limit runs out (a grid of a few small cubes can pass every
    barrier within one tick)."""
    spec = W.cavity(4, 16)
    state = W.initial_state(spec, 5, 1e-2)
    g = gpu_grid(spec, bcm.PREC_F32_REFINE, state)
    g.set_launch(1, 1, persistent=persistent)
    g.set_solver(barrier_timeout_s=1e-9)
    with pytest.raises(bcm.BCMError) as ei:
        g.step(1, rtol=1e-12)
    assert ei.value.status == bcm.BCM_E_TIMEOUT
    g.set_solver(barrier_timeout_s=2.0)
    g.load_state(state)
    g.step(2, rtol=1e-12)
    ost, _ = oracle_run(spec, state, 2, 1e-13)
    compare_fields(g, ost, spec, TOL32, per_component=False)


def two_level_with_bodies():
    """A channel refined 2:1 in all three directions around a fixed sphere and a
    rotating, translating ellipsoid (both inside the refined block)."""
    spec = W.two_level_channel(4, 4, 4, 8, (1, 1, 1), (3, 3, 3), 1 / 16., 0)
    spec.bodies = [[W.Body(W.BODY_SPHERE, np.array([0.9, 1.0, 1.0]), np.array([0.22] * 3)),
                    W.Body(W.BODY_ELLIPSOID, np.array([1.25, 0.9, 1.1]),
                           np.array([0.12, 0.07, 0.09]), np.array([0.9, 0.1, 0.3, 0.3]) /
                           np.linalg.norm([0.9, 0.1, 0.3, 0.3]), np.array([0.4, -1.0, 0.6]),
                           np.array([0.02, 0.0, 0.0]))]]
    return spec


@pytest.mark.parametrize("persistent", [None, 2, 3])
@pytest.mark.parametrize("prec", [bcm.PREC_F64, bcm.PREC_F32_REFINE])
def test_two_level_step(prec, persistent):
    """The full step on a two-level grid: paper halos for momentum, flux-form Poisson
    at the 2:1 faces, bodies in the refined block, against the oracle (default launch
    shape, the single-reduction and the streaming persistent PCG)."""
    spec = two_level_with_bodies()
    state = W.initial_state(spec, seed=23, noise=1e-3)
    ost, ostats = oracle_run(spec, state, 3, 1e-13)
    g = gpu_grid(spec, prec, state)
    if persistent is not None:
        g.set_launch(1, 1, persistent=persistent)
    st = g.step(3, rtol=1e-13 if prec == bcm.PREC_F64 else 1e-12)
    assert st[0]["converged"] == 1
    if prec == bcm.PREC_F64:
        compare_fields(g, ost, spec, TOL64)
        assert abs(st[0]["cg_iters"] - ostats[0]["cg_iters"]) <= 2
        for e in range(3):
            assert abs(st[0]["drag"][e] - ostats[0]["drag"][e]) <= 1e-8 * abs(ostats[0]["drag"][0])
    else:
        compare_fields(g, ost, spec, TOL32, per_component=False)
