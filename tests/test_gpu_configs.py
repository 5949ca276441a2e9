"""The five workloads at their full sizes, in the launch configurations the library
uses: against the oracle where it finishes in seconds (the 64^3 cavity, single sims of
the batch), otherwise by properties that hold at any size (FP64 residual and
divergence at the solver tolerance, mixed against FP64 on the GPU, adjoint against
finite differences of the GPU forward)."""
import numpy as np
import pytest

import oracle as O
from paper_1808_04099_gb300 import workloads as W
from _util import demean_per_sim, oracle_run, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1808_04099_gb300 import adjoint, bcm  # noqa: E402


def velocity(g):
    return np.concatenate([g.numpy(f) for f in (bcm.U, bcm.V, bcm.W)])


def test_cavity_64_ten_steps_fp64_vs_oracle():
    """Lid-driven cavity, 4x4x4 cubes of 16^3, Re 100, 10 steps, seeded noise 1e-3."""
    spec = W.config_cavity64(10)
    state = W.initial_state(spec, seed=0, noise=1e-3)
    ost, ostats = oracle_run(spec, state, 10, 1e-13)
    g = bcm.Grid(spec, bcm.PREC_F64)
    g.load_state(state)
    st = g.step(10, rtol=1e-13)
    ref = np.concatenate([ost[k] for k in ("u", "v", "w")])
    assert rel_l2(velocity(g), ref) <= 1e-10
    assert rel_l2(demean_per_sim(g.numpy(bcm.P), spec), demean_per_sim(ost["p"], spec)) <= 1e-10
    assert st[0]["steps"] == 10 and st[0]["div_rel"] <= 1e-12
    # at the workload's own tolerance the step meets it too
    g2 = bcm.Grid(spec, bcm.PREC_F64)
    g2.load_state(state)
    st2 = g2.step(10, rtol=1e-10)
    assert st2[0]["converged"] == 1 and st2[0]["rel_resid"] <= 1e-10


def test_two_level_83M_cells_mixed_vs_fp64():
    """20,288 cubes of 16^3 on two levels, three rotating ellipsoids (solid fraction
    recomputed every step): one mixed step at residual 1e-8 against the FP64 path."""
    spec = W.config_two_level(1)
    state = W.initial_state(spec)
    g32 = bcm.Grid(spec, bcm.PREC_F32_REFINE)
    g32.load_state(state)
    s32 = g32.step(1, rtol=1e-10)[0]
    assert s32["converged"] == 1 and s32["rel_resid"] <= 1e-10
    vel32 = velocity(g32)
    p32 = g32.numpy(bcm.P)
    del g32
    torch.cuda.empty_cache()
    g64 = bcm.Grid(spec, bcm.PREC_F64)
    g64.load_state(state)
    s64 = g64.step(1, rtol=1e-10)[0]
    assert s64["converged"] == 1
    assert np.all(np.isfinite(vel32))
    assert rel_l2(vel32, velocity(g64)) <= 1e-6
    assert rel_l2(p32, g64.numpy(bcm.P)) <= 1e-6
    assert abs(s32["drag"][0] - s64["drag"][0]) <= 1e-5 * abs(s64["drag"][0])


def test_adjoint_33M_cells_against_gpu_finite_difference():
    """Sphere in 32x16x16 cubes of 16^3 with inflow modes: two steps forward and back;
    dJ/dc_x and dJ/da_1 against central differences of the FP64 GPU forward."""
    spec = W.sphere_channel(32, 16, 16, 16, steps=2)
    modes = np.zeros(8)
    center = np.array([1.0, 1.0, 1.0])
    run = adjoint.AdjointRun(spec, modes, center, 0.25, 2, checkpoint_every=1, rtol=1e-12)
    J = run.forward()
    ga, gc = run.backward()
    del run
    torch.cuda.empty_cache()

    def J_of(m, c):
        r = adjoint.AdjointRun(spec, m, c, 0.25, 2, rtol=1e-12)
        v = r.forward()
        del r
        torch.cuda.empty_cache()
        return v

    h = 1e-4
    e = np.array([h, 0.0, 0.0])
    fd_cx = (J_of(modes, center + e) - J_of(modes, center - e)) / (2 * h)
    m1 = modes.copy()
    m1[0] = h
    fd_a1 = (J_of(m1, center) - J_of(-m1, center)) / (2 * h)
    assert abs(gc[0] - fd_cx) <= 1e-5 * abs(fd_cx)
    assert abs(ga[0] - fd_a1) <= 1e-5 * abs(fd_a1)
    assert J > 0


def test_batched_64_sims_graph_steps():
    """64 cavity / sphere sims with log-uniform cube counts in one flattened grid,
    graph-captured mixed steps; the three smallest sims against their own oracle runs."""
    spec = W.batched_mix(64, seed=0, steps=3)
    state = W.initial_state(spec, seed=1, noise=1e-3)
    g = bcm.Grid(spec, bcm.PREC_F32_REFINE)
    g.load_state(state)
    st = g.step_graph(3, rtol=1e-12)
    assert all(s["converged"] == 1 for s in st)
    sizes = np.diff(spec.sim_cube_offset)
    B3 = spec.B ** 3
    for s in np.argsort(sizes)[:3]:
        a, b = spec.sim_cube_offset[s], spec.sim_cube_offset[s + 1]
        sub = W.concat([W.GridSpec(
            B=spec.B, max_level=spec.max_level,
            sim_cube_offset=np.array([0, b - a], np.int32), cube_ijk=spec.cube_ijk[a:b],
            cube_level=spec.cube_level[a:b], sim_extent=spec.sim_extent[s:s + 1],
            sim_origin=spec.sim_origin[s:s + 1], sim_h0=spec.sim_h0[s:s + 1],
            sim_bc=spec.sim_bc[s:s + 1], sim_bc_vel=spec.sim_bc_vel[s:s + 1],
            sim_nu=spec.sim_nu[s:s + 1], sim_dt=spec.sim_dt[s:s + 1],
            sim_uconv=spec.sim_uconv[s:s + 1], bodies=[spec.bodies[s]],
            inflow_modes=spec.inflow_modes[s:s + 1])])
        slots_all = W.outflow_slots(spec)
        mine = [k for k, (c, f) in enumerate(slots_all) if a <= c < b]
        sub_state = W.State(state.u[a * B3:b * B3], state.v[a * B3:b * B3],
                            state.w[a * B3:b * B3], state.p[a * B3:b * B3],
                            state.ub[mine] if len(mine) else state.ub[:0])
        ost, _ = oracle_run(sub, sub_state, 3, 1e-13)
        vel = np.concatenate([g.numpy(f)[a * B3:b * B3] for f in (bcm.U, bcm.V, bcm.W)])
        ref = np.concatenate([ost[k] for k in ("u", "v", "w")])
        assert rel_l2(vel, ref) <= 1e-6, s
