"""The multigrid preconditioner on the GPU (BCM_PRECOND_MULTIGRID) against the oracle:
one V-cycle z = M^-1 r against the oracle's V-cycle built from its definition (Galerkin
products of the oracle's own operator) on single-level and two-level grids (2:1 faces
on every per-cube level, the refined cubes aggregated first), and whole steps with the
multigrid-preconditioned PCG, eager and captured in graph steps (conditional loops),
against the oracle's steps (whose Jacobi-PCG reaches the same unique solution)."""
import numpy as np
import pytest

import oracle as O
from oracle import mg_oracle as MGO
from paper_1808_04099_gb300 import workloads as W
from _util import assert_close, demean_per_sim, oracle_run, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1808_04099_gb300 import bcm  # noqa: E402

TOL64, TOL32 = 1e-10, 1e-6

GRIDS = {
    "channel_B4": lambda: W.sphere_channel(4, 2, 2, 4, length=(4.0, 2.0, 2.0), radius=0.3),
    "cavity_B8": lambda: W.cavity(2, 8),
    "periodic_B4": lambda: W.periodic_box(2, 4),
    "channel_B16": lambda: W.sphere_channel(2, 1, 1, 16, length=(2.0, 1.0, 1.0), radius=0.2,
                                            center=(0.6, 0.5, 0.5)),
    "batched": lambda: W.concat([W.cavity(2, 4, re=300.0),
                                 W.sphere_channel(4, 2, 2, 4, radius=0.3),
                                 W.cavity(3, 4, re=700.0)]),
    # a level-0 row whose first cube is refined: per-cell levels only (B = 4), the
    # tile levels at 8^3 (B = 8) and at 16^3 and 8^3 (B = 16)
    "two_level_B4": lambda: W.two_level_channel(3, 1, 1, 4, (0, 0, 0), (1, 1, 1), 1 / 8., 0),
    "two_level_B8": lambda: W.two_level_channel(2, 1, 1, 8, (0, 0, 0), (1, 1, 1), 1 / 16., 0),
    "two_level_B16": lambda: W.two_level_channel(2, 1, 1, 16, (1, 0, 0), (2, 1, 1), 1 / 32., 0),
    "two_level_3d_B4": lambda: W.two_level_channel(4, 2, 2, 4, (1, 0, 0), (3, 2, 2), 1 / 8., 0),
}


@pytest.mark.parametrize("name", sorted(GRIDS))
def test_vcycle_matches_oracle(name):
    spec = GRIDS[name]()
    g = bcm.Grid(spec, bcm.PREC_F64)
    mg = MGO.MG(O.Oracle(spec))
    rng = np.random.default_rng(7)
    for _ in range(2):
        r = rng.standard_normal(spec.n_cells)
        z = g.apply_preconditioner(r).cpu().numpy()
        ref = mg.apply(r)
        assert rel_l2(z, ref) <= 1e-12


def velocity(g):
    return np.concatenate([g.numpy(f) for f in (bcm.U, bcm.V, bcm.W)])


def check(g, ost, spec, tol):
    ref = np.concatenate([ost[k] for k in ("u", "v", "w")])
    assert_close(velocity(g), ref, g.numpy(bcm.P), ost["p"], spec, tol)


@pytest.mark.parametrize("prec", [bcm.PREC_F64, bcm.PREC_F32_REFINE])
def test_mg_steps_match_oracle(prec):
    """Sphere flow (B = 8) and a batch of ragged sims: two steps with the multigrid PCG
    against the oracle; fewer PCG iterations than the Jacobi PCG on the same step."""
    for spec in (W.sphere_channel(4, 2, 2, 8, radius=0.3),
                 W.concat([W.cavity(2, 8, re=250.0), W.sphere_channel(4, 2, 2, 8, radius=0.3)]),
                 two_level_bodies()):
        state = W.initial_state(spec, seed=51, noise=1e-3)
        ost, ostats = oracle_run(spec, state, 2, 1e-13)
        rtol = 1e-13 if prec == bcm.PREC_F64 else 1e-12
        g = bcm.Grid(spec, prec)
        g.load_state(state)
        g.set_preconditioner(bcm.PRECOND_MULTIGRID)
        st = g.step(2, rtol=rtol)
        assert all(s["converged"] == 1 and s["pcg_form"] == 4 for s in st)
        check(g, ost, spec, TOL64 if prec == bcm.PREC_F64 else TOL32)
        if prec == bcm.PREC_F64:
            for s, o in zip(st, ostats):
                assert s["cg_iters"] * 2 < o["cg_iters"], (s["cg_iters"], o["cg_iters"])


def test_mg_full_size_sphere_mixed():
    """The 4.19M-cell sphere flow, two mixed steps at residual 1e-10 with the multigrid
    PCG: converged, divergence at the residual, and within 1e-6 of the Jacobi PCG."""
    spec = W.config_sphere(2)
    state = W.initial_state(spec)
    runs = []
    for kind in (bcm.PRECOND_MULTIGRID, bcm.PRECOND_JACOBI):
        g = bcm.Grid(spec, bcm.PREC_F32_REFINE)
        g.load_state(state)
        g.set_preconditioner(kind)
        st = g.step(2, rtol=1e-10)
        assert st[0]["converged"] == 1 and st[0]["rel_resid"] <= 1e-10
        assert st[0]["div_rel"] <= 1e-9
        runs.append((velocity(g), st[0]["cg_iters"]))
        del g
        torch.cuda.empty_cache()
    assert rel_l2(runs[0][0], runs[1][0]) <= TOL32
    assert runs[0][1] * 4 < runs[1][1], (runs[0][1], runs[1][1])


def two_level_bodies():
    """4x2x2 coarse cubes of 8^3, the middle 2x2x2 refined (72 cubes, 36,864 cells),
    one seeded rotating ellipsoid in the refined block, inflow and outflow."""
    return W.two_level_channel(4, 2, 2, 8, (1, 0, 0), (3, 2, 2), 1 / 16., 1, seed=3)


GRAPH_GRIDS = {
    "sphere_B8": lambda: W.sphere_channel(4, 2, 2, 8, radius=0.3),
    "two_level": two_level_bodies,
    "batched": lambda: W.concat([two_level_bodies(),
                                 W.two_level_channel(2, 1, 1, 8, (0, 0, 0), (1, 1, 1), 1 / 16., 0,
                                                     re=400.0)]),
}


@pytest.mark.parametrize("name", sorted(GRAPH_GRIDS))
@pytest.mark.parametrize("prec", [bcm.PREC_F64, bcm.PREC_F32_REFINE])
def test_mg_graph_steps_match_oracle_and_eager(name, prec):
    """Graph-captured steps with the multigrid PCG (its loops as conditional nodes)
    against the oracle, and against eager steps: the same iterations, the launches
    inside the loops counted."""
    spec = GRAPH_GRIDS[name]()
    state = W.initial_state(spec, seed=52, noise=1e-3)
    steps = 3
    ost, _ = oracle_run(spec, state, steps, 1e-13)
    rtol = 1e-13 if prec == bcm.PREC_F64 else 1e-12
    runs = {}
    for graph in (True, False):
        g = bcm.Grid(spec, prec)
        g.load_state(state)
        g.set_preconditioner(bcm.PRECOND_MULTIGRID)
        g.profile_read(reset=True)
        st = g.step_graph(steps, rtol=rtol) if graph else g.step(steps, rtol=rtol)
        assert all(s["converged"] == 1 and s["pcg_form"] == 4 for s in st), st
        check(g, ost, spec, TOL64 if prec == bcm.PREC_F64 else TOL32)
        _, launches = g.profile_read(reset=True)
        runs[graph] = (velocity(g), [s["cg_iters"] for s in st], launches)
        del g
    assert rel_l2(runs[True][0], runs[False][0]) <= (1e-12 if prec == bcm.PREC_F64 else 1e-7)
    assert runs[True][1] == runs[False][1]
    # the eager solve issues its iterations in batches between flag reads, so it may
    # launch a few iterations more than the loops run
    assert 0.5 * runs[False][2] <= runs[True][2] <= 1.1 * runs[False][2], (runs[True][2],
                                                                          runs[False][2])


def test_mg_two_level_fewer_iterations_than_jacobi():
    """The refined channel's pressure solve: the multigrid PCG needs a fraction of the
    Jacobi PCG's iterations and reaches the same solution."""
    spec = two_level_bodies()
    rng = np.random.default_rng(53)
    b = rng.standard_normal(spec.n_cells)
    out = {}
    for kind in (bcm.PRECOND_MULTIGRID, bcm.PRECOND_JACOBI):
        g = bcm.Grid(spec, bcm.PREC_F64)
        g.set_preconditioner(kind)
        g.field(bcm.RHS).copy_(torch.from_numpy(b))
        g.field(bcm.P).zero_()
        st = g.solve_pressure(1e-12)[0]
        assert st["converged"] == 1
        out[kind] = (demean_per_sim(g.numpy(bcm.P), spec), st["cg_iters"])
    assert rel_l2(out[bcm.PRECOND_MULTIGRID][0], out[bcm.PRECOND_JACOBI][0]) <= 1e-9
    assert out[bcm.PRECOND_MULTIGRID][1] * 4 < out[bcm.PRECOND_JACOBI][1], out
