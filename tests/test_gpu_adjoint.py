"""The discrete adjoint of the step against central finite differences of the FP64
oracle: gradient of the time-averaged drag on a fixed sphere with respect to the eight
inflow-profile amplitudes and the sphere centre, through checkpoint-and-recompute."""
import numpy as np
import pytest

import oracle as O
from paper_1808_04099_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1808_04099_gb300 import adjoint  # noqa: E402

RADIUS = 0.3
STEPS = 4


def base_spec():
    return W.sphere_channel(4, 2, 2, 8, radius=RADIUS, center=(1.0, 1.0, 1.0), re=100.0)


def oracle_J(modes, center):
    spec = base_spec()
    spec.inflow_modes = np.asarray(modes, np.float64)[None, :].copy()
    spec.bodies = [[W.Body(W.BODY_SPHERE, np.asarray(center, np.float64),
                           np.array([RADIUS] * 3))]]
    o = O.Oracle(spec)
    st = o.new_state(W.initial_state(spec))
    J = 0.0
    for _ in range(STEPS):
        stats, rc = o.step(st, 1, rtol=1e-13)
        assert rc == 0
        J += stats[0]["drag"][0] / STEPS
    return J


def test_adjoint_gradient_matches_finite_differences():
    rng = np.random.default_rng(51)
    modes = rng.uniform(-0.05, 0.05, 8)
    center = np.array([1.02, 0.97, 1.05])
    run = adjoint.AdjointRun(base_spec(), modes, center, RADIUS, STEPS, checkpoint_every=2,
                             rtol=1e-13)
    J = run.forward()
    ga, gc = run.backward()
    J0 = oracle_J(modes, center)
    assert abs(J - J0) <= 1e-9 * abs(J0)
    h = 1e-4
    fd = np.zeros(11)
    theta = np.concatenate([modes, center])
    for q in range(11):
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        fd[q] = (oracle_J(tp[:8], tp[8:]) - oracle_J(tm[:8], tm[8:])) / (2 * h)
    g = np.concatenate([ga, gc])
    err = np.linalg.norm(g - fd) / np.linalg.norm(fd)
    print(f"adjoint vs central FD (h={h}): relative error {err:.3e}")
    assert err <= 1e-5, (err, g, fd)


def test_adjoint_through_autograd_and_checkpoint_independence():
    spec = base_spec()
    a = torch.zeros(8, dtype=torch.float64, requires_grad=True)
    c = torch.tensor([1.0, 1.0, 1.0], dtype=torch.float64, requires_grad=True)
    J = adjoint.drag(a, c, spec, RADIUS, STEPS, checkpoint_every=1, rtol=1e-13)
    J.backward()
    run = adjoint.AdjointRun(spec, np.zeros(8), np.ones(3), RADIUS, STEPS, checkpoint_every=4,
                             rtol=1e-13)
    J2 = run.forward()
    ga, gc = run.backward()
    assert abs(float(J.detach()) - J2) <= 1e-12 * abs(J2)
    g1 = np.concatenate([a.grad.numpy(), c.grad.numpy()])
    g2 = np.concatenate([ga, gc])
    assert np.linalg.norm(g1 - g2) <= 1e-10 * np.linalg.norm(g2)
    # symmetry of the problem: no lateral force gradient in y at the symmetric point
    # (the inflow modes break it, so only the centre-y/z derivative is ~0 at a = 0)
    assert abs(c.grad[1].item()) <= 1e-8 * abs(c.grad[0].item()) + 1e-12


def test_adjoint_amplitude_gradient_at_zero_amplitudes():
    """At a = 0 the inflow profile is flat, yet dJ/da is not zero: the adjoint must
    differentiate through the profile factor there too."""
    modes = np.zeros(8)
    center = np.array([1.0, 1.0, 1.0])
    run = adjoint.AdjointRun(base_spec(), modes, center, RADIUS, STEPS, checkpoint_every=2,
                             rtol=1e-13)
    run.forward()
    ga, gc = run.backward()
    h = 1e-4
    # modes (1,1) and (1,3) are symmetric about the channel centre (non-zero response);
    # (2,2) is antisymmetric, so its first-order effect on the drag vanishes there
    for m in (0, 4, 3):
        tp = modes.copy()
        tp[m] = h
        fd = (oracle_J(tp, center) - oracle_J(-tp, center)) / (2 * h)
        assert abs(ga[m] - fd) <= 1e-5 * abs(fd) + 1e-12, (m, ga[m], fd)
    assert abs(ga[0]) > 1e-3


def test_adjoint_gradient_matches_taped_oracle():
    """The GPU adjoint against reverse-mode autograd of the taped restatement of the
    step (oracle/taped.py: one array per field, dense Poisson solve) on a 1,024-cell
    channel: both are exact derivatives of the same discrete FP64 step, so they agree
    to the solver tolerance."""
    from oracle import taped as T
    modes = np.array([0.03, -0.02, 0.015, 0.01, -0.025, 0.02, -0.01, 0.005])
    center = np.array([0.97, 0.52, 0.46])
    radius, steps = 0.25, 3
    spec = W.sphere_channel(2, 1, 1, 8, length=(2.0, 1.0, 1.0), radius=radius,
                            center=tuple(center), re=100.0)
    Jt, ta, tcg = T.drag_gradient(spec, modes, center, radius, steps)
    run = adjoint.AdjointRun(spec, modes, center, radius, steps, checkpoint_every=2,
                             rtol=1e-13)
    J = run.forward()
    ga, gc = run.backward()
    assert abs(J - Jt) <= 1e-11 * abs(Jt)
    g, t = np.concatenate([ga, gc]), np.concatenate([ta, tcg])
    assert np.linalg.norm(g - t) <= 1e-8 * np.linalg.norm(t), (g, t)


def test_drag_mean_is_the_mean_of_the_steps_drag():
    """bcm_drag_mean (the adjoint's objective J in the library) against the mean of the
    per-step drag the steps report, for every sim of a batch; a reset starts anew."""
    from paper_1808_04099_gb300 import bcm
    spec = W.concat([W.sphere_channel(2, 1, 1, 8, length=(2.0, 1.0, 1.0), radius=0.25,
                                      center=(0.7, 0.5, 0.5), re=100.0),
                     W.sphere_channel(4, 2, 2, 8, radius=0.3)])
    g = bcm.Grid(spec, bcm.PREC_F64)
    g.load_state(W.initial_state(spec, seed=62, noise=1e-3))
    assert np.all(g.drag_mean(reset=True) == 0.0)
    drags = []
    for _ in range(4):
        st = g.step(1, rtol=1e-12)
        drags.append([s["drag"] for s in st])
    ref = np.mean(np.asarray(drags), axis=0)
    got = g.drag_mean(reset=True)
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()
    st = g.step(1, rtol=1e-12)
    got = g.drag_mean()
    assert np.abs(got - np.asarray([s["drag"] for s in st])).max() <= 1e-15 * np.abs(got).max()
