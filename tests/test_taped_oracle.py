"""Pins of the taped restatement of the step (oracle/taped.py), the gradient oracle of the
adjoint (R14): its forward equals the C oracle's steps on the same channel (drag per
step, velocity, pressure, outflow face values), and its autograd gradient of the
time-averaged drag with respect to the eight inflow amplitudes and the sphere centre
equals central differences of the C oracle.  The two restatements share no code: the
C oracle works cube by cube with halo rules and PCG, the taped one on one array with
shifts and a dense solve."""
import numpy as np
import pytest

import oracle as O
from paper_1808_04099_gb300 import workloads as W

torch = pytest.importorskip("torch")
from oracle import taped as T  # noqa: E402

RADIUS = 0.25
STEPS = 3
MODES = np.array([0.03, -0.02, 0.015, 0.01, -0.025, 0.02, -0.01, 0.005])
CENTER = np.array([0.97, 0.52, 0.46])


def spec_with(modes, center):
    spec = W.sphere_channel(2, 1, 1, 8, length=(2.0, 1.0, 1.0), radius=RADIUS,
                            center=tuple(center), re=100.0)
    spec.inflow_modes = np.asarray(modes, np.float64)[None, :].copy()
    spec.bodies = [[W.Body(W.BODY_SPHERE, np.asarray(center, np.float64),
                           np.array([RADIUS] * 3))]]
    return spec


def oracle_run(modes, center, steps=STEPS):
    spec = spec_with(modes, center)
    o = O.Oracle(spec)
    st = o.new_state(W.initial_state(spec))
    drags = []
    for _ in range(steps):
        stats, rc = o.step(st, 1, rtol=1e-14)
        assert rc == 0
        drags.append(stats[0]["drag"])
    return np.array(drags), st, spec


def test_taped_forward_equals_c_oracle():
    drags, st, spec = oracle_run(MODES, CENTER)
    tc = T.TapedChannel(spec)
    J, drag, (u, v, w, p), ub = tc.run(MODES, CENTER, RADIUS, STEPS, W.initial_state(spec))
    # the C oracle's PCG runs to 1e-14: both sides agree to rounding (~1e-15 here)
    assert np.allclose(drag.numpy(), drags, rtol=1e-12, atol=1e-14)
    assert abs(float(J) - drags[:, 0].mean()) <= 1e-12 * abs(drags[:, 0].mean())
    for got, key in ((u, "u"), (v, "v"), (w, "w")):
        want = tc.to_grid(st[key])
        assert np.abs(got.numpy() - want).max() <= 1e-12 * np.abs(want).max(), key
    want_p = tc.to_grid(st["p"])
    assert np.abs(p.numpy() - want_p).max() <= 1e-12 * np.abs(want_p).max()
    assert np.allclose(ub.numpy(), tc.ub_to_grid(st["ub"]), rtol=0, atol=1e-12)


def test_taped_gradient_equals_oracle_central_differences():
    J, ga, gc = T.drag_gradient(spec_with(MODES, CENTER), MODES, CENTER, RADIUS, STEPS)
    theta = np.concatenate([MODES, CENTER])
    hstep = 1e-4
    fd = np.zeros(11)
    for q in range(11):
        tp, tm = theta.copy(), theta.copy()
        tp[q] += hstep
        tm[q] -= hstep
        Jp = oracle_run(tp[:8], tp[8:])[0][:, 0].mean()
        Jm = oracle_run(tm[:8], tm[8:])[0][:, 0].mean()
        fd[q] = (Jp - Jm) / (2 * hstep)
    g = np.concatenate([ga, gc])
    assert np.linalg.norm(fd) > 1e-3  # the drag does depend on the parameters
    err = np.linalg.norm(g - fd) / np.linalg.norm(fd)
    assert err <= 1e-6, (err, g, fd)


def test_taped_gradient_direction_equals_its_own_difference_quotient():
    """Reverse mode against a central difference of the taped forward along a random
    direction (no solver tolerance on either side: the dense solve is exact)."""
    spec = spec_with(MODES, CENTER)
    tc = T.TapedChannel(spec)
    st = W.initial_state(spec)
    _, ga, gc = T.drag_gradient(spec, MODES, CENTER, RADIUS, STEPS)
    rng = np.random.default_rng(5)
    dirn = rng.standard_normal(11)
    eps = 1e-5
    theta = np.concatenate([MODES, CENTER])

    def J(t):
        return float(tc.run(t[:8], t[8:], RADIUS, STEPS, st)[0])

    fd = (J(theta + eps * dirn) - J(theta - eps * dirn)) / (2 * eps)
    assert abs(np.dot(np.concatenate([ga, gc]), dirn) - fd) <= 1e-7 * abs(fd)
