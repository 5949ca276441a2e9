"""GPU parity of the fused single-barrier PCG (bcm_stats.pcg_form 5, launch shape
persistent = 5), an inner solve of mixed precision on 16^3 cubes: against the FP64 oracle on grids that cover
every kind of face (same level, domain walls, outflow, periodic wrap, 2:1 in both
directions) and batched sims, against the two-pass streaming form at the benchmark's
full size, inside captured steps, and its bounded waits and iteration limit.

Tolerances as in test_gpu_parity: mixed steps within 1e-6 (relative L2 of the velocity
vector and of the pressure), both sides solving tighter than that."""
import numpy as np
import pytest

from paper_1808_04099_gb300 import workloads as W
from _util import demean_per_sim, oracle_run, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1808_04099_gb300 import bcm  # noqa: E402

TOL32 = 1e-6
FUSED = 5


def grid(spec, state, prec=bcm.PREC_F32_REFINE):
    g = bcm.Grid(spec, prec)
    g.load_state(state)
    g.set_launch(1, 1, persistent=FUSED)
    return g


def errors(g, ost, spec):
    vel = np.concatenate([g.numpy(f) for f in (bcm.U, bcm.V, bcm.W)])
    ref = np.concatenate([ost[k] for k in ("u", "v", "w")])
    ev = rel_l2(vel, ref)
    ep = rel_l2(demean_per_sim(g.numpy(bcm.P), spec), demean_per_sim(ost["p"], spec))
    # largest cell error against the largest value: an error confined to a few cells
    # (a face, the 2:1 interface, the body shell) cannot hide in the norm
    mv = np.max(np.abs(vel - ref)) / np.max(np.abs(ref))
    return ev, ep, mv


def two_level_b16():
    """4x2x2 coarse cubes of 16^3, the middle 2x2x2 refined (72 cubes, 294,912 cells),
    a fixed sphere and a rotating ellipsoid in the refined block."""
    spec = W.two_level_channel(4, 2, 2, 16, (1, 0, 0), (3, 2, 2), 1 / 32., 0)
    spec.bodies = [[W.Body(W.BODY_SPHERE, np.array([1.0, 0.5, 0.5]), np.array([0.15] * 3)),
                    W.Body(W.BODY_ELLIPSOID, np.array([1.3, 0.55, 0.45]),
                           np.array([0.08, 0.05, 0.06]),
                           np.array([0.9, 0.1, 0.3, 0.3]) / np.linalg.norm([0.9, 0.1, 0.3, 0.3]),
                           np.array([0.4, -1.0, 0.6]), np.zeros(3))]]
    return spec


CASES = {
    "sphere_2x1x1": lambda: W.sphere_channel(2, 1, 1, 16, length=(2.0, 1.0, 1.0), radius=0.2,
                                             center=(0.6, 0.5, 0.5)),
    "sphere_4x2x2": lambda: W.sphere_channel(4, 2, 2, 16, length=(2.0, 1.0, 1.0), radius=0.2,
                                             center=(0.6, 0.5, 0.5)),
    "cavity_2": lambda: W.cavity(2, 16),
    "periodic_2": lambda: W.periodic_box(2, 16),
    "two_level": two_level_b16,
    "batched": lambda: W.concat([W.cavity(2, 16, re=300.0),
                                 W.sphere_channel(2, 1, 1, 16, length=(2.0, 1.0, 1.0),
                                                  radius=0.2, center=(0.6, 0.5, 0.5)),
                                 W.cavity(1, 16, re=150.0)]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fused_mixed_steps_against_oracle(name):
    spec = CASES[name]()
    state = W.initial_state(spec, seed=41, noise=1e-3)
    nsteps = 3
    ost, _ = oracle_run(spec, state, nsteps, 1e-13)
    g = grid(spec, state)
    st = g.step(nsteps, rtol=1e-12)
    assert all(s["pcg_form"] == FUSED for s in st)
    assert all(s["converged"] == 1 and s["rel_resid"] <= 1e-12 for s in st)
    ev, ep, mv = errors(g, ost, spec)
    assert ev <= TOL32 and ep <= TOL32, (ev, ep)
    assert mv <= 1e-5, mv


def test_fused_pressure_solve_against_oracle():
    """A bare pressure solve of a random right-hand side: the fused FP32 inner PCG in
    FP64 defect correction reaches the oracle's FP64 solution."""
    import oracle as O
    spec = two_level_b16()
    rng = np.random.default_rng(43)
    b = rng.standard_normal(spec.n_cells)
    o = O.Oracle(spec)
    x_ref, _, rc = o.solve_pressure(b, rtol=1e-13)
    assert rc == 0
    g = bcm.Grid(spec, bcm.PREC_F32_REFINE)
    g.set_launch(1, 1, persistent=FUSED)
    g.field(bcm.RHS).copy_(torch.from_numpy(b))
    g.field(bcm.P).zero_()
    st = g.solve_pressure(1e-12)
    assert st[0]["pcg_form"] == FUSED and st[0]["converged"] == 1
    assert rel_l2(g.numpy(bcm.P), x_ref) <= 1e-9


def test_fused_against_streaming_full_size():
    """The 4.19M-cell sphere flow: two mixed steps with the fused form and with the
    two-pass streaming form agree."""
    spec = W.config_sphere(2)
    state = W.initial_state(spec)
    out = {}
    for persistent in (5, 1):
        g = grid(spec, state)
        g.set_launch(1, 1, persistent=persistent)
        st = g.step(2, rtol=1e-10)[0]
        assert st["pcg_form"] == persistent and st["converged"] == 1
        assert st["rel_resid"] <= 1e-10 and st["div_rel"] <= 1e-9
        out[persistent] = (np.concatenate([g.numpy(f) for f in (bcm.U, bcm.V, bcm.W)]),
                           g.numpy(bcm.P), st["cg_iters"])
        del g
    assert rel_l2(out[5][0], out[1][0]) <= TOL32
    assert rel_l2(out[5][1], out[1][1]) <= TOL32
    # the same iterates in exact arithmetic within one inner solve; across defect-
    # correction cycles the fused form resumes its direction from the stored r and p
    # (measured: 17 % fewer inner iterations over the two steps), never many more
    assert 0.5 * out[1][2] <= out[5][2] <= 1.1 * out[1][2]


def test_fused_graph_steps_match_eager_and_oracle():
    spec = CASES["sphere_4x2x2"]()
    state = W.initial_state(spec, seed=44, noise=1e-3)
    ost, _ = oracle_run(spec, state, 3, 1e-13)
    g = grid(spec, state)
    st = g.step_graph(3, rtol=1e-12)
    assert st[0]["pcg_form"] == FUSED and st[0]["converged"] == 1
    ev, ep, _ = errors(g, ost, spec)
    assert ev <= TOL32 and ep <= TOL32


def test_fused_barrier_timeout_reported_and_recovered():
    """A 1 ns limit on the grid barrier and the copy waits ends the solve with
    BCM_E_TIMEOUT; the next solve with the normal limit is exact."""
    spec = W.cavity(4, 16)
    state = W.initial_state(spec, 5, 1e-2)
    g = grid(spec, state)
    g.set_solver(barrier_timeout_s=1e-9)
    with pytest.raises(bcm.BCMError) as ei:
        g.step(1, rtol=1e-12)
    assert ei.value.status == bcm.BCM_E_TIMEOUT
    g.set_solver(barrier_timeout_s=2.0)
    g.load_state(state)
    st = g.step(2, rtol=1e-12)
    assert st[0]["pcg_form"] == FUSED
    ost, _ = oracle_run(spec, state, 2, 1e-13)
    ev, ep, _ = errors(g, ost, spec)
    assert ev <= TOL32 and ep <= TOL32


def test_fused_iteration_limit():
    spec = CASES["sphere_2x1x1"]()
    state = W.initial_state(spec, seed=45, noise=1e-3)
    g = grid(spec, state)
    g.set_solver(max_cycles=1)
    with pytest.raises(bcm.BCMError) as ei:
        g.step(1, rtol=1e-14, max_iter=3)
    assert ei.value.status == bcm.BCM_E_NOT_CONVERGED
