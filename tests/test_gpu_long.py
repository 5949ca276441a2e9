"""Parity over the workloads' own horizons, on scaled-down instances the oracle runs in
seconds (the full sizes are covered in test_gpu_configs and test_gpu_parity):

* the sphere flow over 200 steps (its step count), FP64 within 1e-10 of the oracle and
  the FP32 Poisson sweeps inside FP64 defect correction within 1e-6 on an FP64 state;
  with an FP32 state the error after 200 steps is the flow's own amplification of the
  per-step rounding of the state (measured: ~3e-4 against 1e-6), which a test bounds
  by the FP64 path's divergence from one such rounding;
* the two-level grid with three rotating ellipsoids (solid fraction recomputed every
  step) over 20 steps, FP64 and the mixed pressure solve on an FP64 state, and the
  FP32-state path against its amplification bound;
* the adjoint over 50 steps with a checkpoint every 10, all eleven gradient components
  (eight inflow amplitudes, three centre coordinates) against central differences of the
  oracle.

Every comparison also bounds the largest cell error (tests/_util.assert_close)."""
import numpy as np
import pytest

import oracle as O
from paper_1808_04099_gb300 import workloads as W
from _util import assert_close, oracle_run, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1808_04099_gb300 import adjoint, bcm  # noqa: E402

TOL64 = 1e-10
TOL32 = 1e-6


def velocity(g):
    return np.concatenate([g.numpy(f) for f in (bcm.U, bcm.V, bcm.W)])


def run_both(spec, state, steps, precs=((bcm.PREC_F64, 1e-13, TOL64),
                                         (bcm.PREC_F64_REFINE, 1e-12, TOL32))):
    ost, _ = oracle_run(spec, state, steps, 1e-13)
    ref = np.concatenate([ost[k] for k in ("u", "v", "w")])
    out = {}
    for prec, rtol, tol in precs:
        g = bcm.Grid(spec, prec)
        g.load_state(state)
        st = g.step(steps, rtol=rtol)
        assert all(s["converged"] == 1 and s["steps"] == steps for s in st)
        out[prec] = assert_close(velocity(g), ref, g.numpy(bcm.P), ost["p"], spec, tol)
        print(f"{spec.name} {steps} steps prec {prec}: rel L2 u {out[prec][0]:.2e} "
              f"p {out[prec][1]:.2e}, largest cell u {out[prec][2]:.2e} p {out[prec][3]:.2e}")
        del g
    return out


def test_sphere_flow_200_steps_against_oracle():
    """The sphere flow's 200 steps on 4x2x2 cubes of 8^3 (same domain, body, Re 300)."""
    spec = W.sphere_channel(4, 2, 2, 8, radius=0.3)
    run_both(spec, W.initial_state(spec, seed=3, noise=1e-3), 200)


def two_level_rotating():
    """8x4x4 coarse cubes of 8^3 on [0,4]x[0,2]x[0,2], the 4x2x2 middle ones refined once
    (240 cubes, 122,880 cells), three ellipsoids with seeded semi-axes, centres, angular
    velocities and orientations inside the refined block, Re 1000."""
    spec = W.two_level_channel(8, 4, 4, 8, (2, 1, 1), (6, 3, 3), 1.0 / 16.0, 0, 0, 1000.0)
    rng = np.random.default_rng(0)
    bodies = []
    for _ in range(3):
        ax = rng.uniform(0.06, 0.15, 3)
        cen = rng.uniform([1.3, 0.75, 0.75], [2.7, 1.25, 1.25])
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        bodies.append(W.Body(W.BODY_ELLIPSOID, cen, ax, q, axis * rng.uniform(0.5, 2.0),
                             np.zeros(3)))
    spec.bodies = [bodies]
    return spec


def test_two_level_rotating_ellipsoids_20_steps_against_oracle():
    spec = two_level_rotating()
    state = W.initial_state(spec, seed=4, noise=1e-3)
    run_both(spec, state, 20)
    # the FP32 state: velocity within 1e-6 too (measured 2e-7); its pressure, a small
    # field on this grid, moves by ~7e-6 with the state's FP32 rounding, which the FP64
    # state above removes
    ost, _ = oracle_run(spec, state, 20, 1e-13)
    g32 = bcm.Grid(spec, bcm.PREC_F32_REFINE)
    g32.load_state(state)
    g32.step(20, rtol=1e-12)
    ref = np.concatenate([ost[k] for k in ("u", "v", "w")])
    assert rel_l2(velocity(g32), ref) <= TOL32


def test_adjoint_50_steps_checkpoint_10_all_components_against_oracle():
    """dJ/d(a_1..a_8, c) of the time-averaged drag over 50 steps, checkpoints every 10
    steps with recompute, against central differences (h = 1e-4) of the oracle."""
    radius, steps = 0.3, 50
    rng = np.random.default_rng(52)
    modes = rng.uniform(-0.05, 0.05, 8)
    center = np.array([1.02, 0.97, 1.03])

    def spec_for(m, c):
        spec = W.sphere_channel(4, 2, 2, 8, radius=radius, center=tuple(c), re=100.0)
        spec.inflow_modes = np.asarray(m, np.float64)[None, :].copy()
        spec.bodies = [[W.Body(W.BODY_SPHERE, np.asarray(c, np.float64), np.array([radius] * 3))]]
        return spec

    def oracle_J(m, c):
        spec = spec_for(m, c)
        o = O.Oracle(spec)
        st = o.new_state(W.initial_state(spec))
        J = 0.0
        for _ in range(steps):
            stats, rc = o.step(st, 1, rtol=1e-13)
            assert rc == 0
            J += stats[0]["drag"][0] / steps
        return J

    run = adjoint.AdjointRun(spec_for(modes, center), modes, center, radius, steps,
                             checkpoint_every=10, rtol=1e-13)
    J = run.forward()
    ga, gc = run.backward()
    assert abs(J - oracle_J(modes, center)) <= 1e-9 * abs(J)
    h = 1e-4
    theta = np.concatenate([modes, center])
    fd = np.zeros(11)
    for q in range(11):
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        fd[q] = (oracle_J(tp[:8], tp[8:]) - oracle_J(tm[:8], tm[8:])) / (2 * h)
    g = np.concatenate([ga, gc])
    err = np.abs(g - fd) / np.linalg.norm(fd)
    print("adjoint 50 steps: per-component error / |fd|:", np.array2string(err, precision=2))
    assert np.linalg.norm(g - fd) <= 1e-5 * np.linalg.norm(fd), (g, fd)
    assert np.all(err <= 1e-5), err


def test_fp64_state_with_fp32_poisson_sweeps_200_steps_within_1e6():
    """BCM_PREC_F64_REFINE: the FP32 inner PCG inside FP64 defect correction (the mixed
    pressure solve) on an FP64 state.  Over the sphere flow's 200 steps it stays within
    1e-6 of the oracle, which the FP32 state cannot: rounding the state to FP32 every
    step is a perturbation of ~3e-8 that this unsteady wake amplifies."""
    spec = W.sphere_channel(4, 2, 2, 8, radius=0.3)
    state = W.initial_state(spec, seed=3, noise=1e-3)
    ost, _ = oracle_run(spec, state, 200, 1e-13)
    ref = np.concatenate([ost[k] for k in ("u", "v", "w")])
    g = bcm.Grid(spec, bcm.PREC_F64_REFINE)
    g.load_state(state)
    st = g.step(200, rtol=1e-12)
    assert st[0]["converged"] == 1 and st[0]["refine_cycles"] >= 1
    assert g.field(bcm.U).dtype == torch.float64
    ev, ep, mv, mp = assert_close(velocity(g), ref, g.numpy(bcm.P), ost["p"], spec, TOL32)
    print(f"F64 state + FP32 Poisson sweeps, 200 steps: rel L2 u {ev:.2e} p {ep:.2e}")


def test_fp32_state_long_horizon_error_is_the_flows_amplification():
    """The FP32-state mixed path over 200 steps against the FP64 path started from the
    FP32-rounded initial state: the flow's own amplification of one FP32 rounding of the
    state.  The mixed path rounds the state (and rounds its FP32 arithmetic) every step,
    and each of those perturbations grows over the steps that follow, so its error is at
    most the step count times that amplified rounding (measured: 53 times; a wrong stencil
    or solve would be O(1))."""
    spec = W.sphere_channel(4, 2, 2, 8, radius=0.3)
    state = W.initial_state(spec, seed=3, noise=1e-3)
    steps = 200
    ost, _ = oracle_run(spec, state, steps, 1e-13)
    ref = np.concatenate([ost[k] for k in ("u", "v", "w")])
    rounded = W.State(*(np.asarray(a, np.float32).astype(np.float64)
                        for a in (state.u, state.v, state.w, state.p)),
                      np.asarray(state.ub, np.float32).astype(np.float64))
    g64 = bcm.Grid(spec, bcm.PREC_F64)
    g64.load_state(rounded)
    g64.step(steps, rtol=1e-13)
    amp = max(np.linalg.norm(velocity(g64) - ref) / np.linalg.norm(ref), 1e-12)
    g32 = bcm.Grid(spec, bcm.PREC_F32_REFINE)
    g32.load_state(state)
    st = g32.step(steps, rtol=1e-12)
    assert st[0]["converged"] == 1
    err = np.linalg.norm(velocity(g32) - ref) / np.linalg.norm(ref)
    print(f"FP32 state, 200 steps: rel L2 {err:.2e}; one rounding amplified: {amp:.2e}")
    assert err <= steps * amp, (err, amp)
