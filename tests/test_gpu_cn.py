"""QUICK + Crank-Nicolson momentum on the GPU (bcm_set_momentum_scheme) against the oracle
(R20 in oracle/bcm_oracle.c): whole steps on grids with every boundary kind, a two-level
grid (the two-layer 2:1 halo QUICK reads), batched sims, graph-captured steps, the
particle IB on top, and the switch back to Adams-Bashforth; the full-size sphere flow in
mixed precision against FP64 on the GPU.  The oracle iterates the Crank-Nicolson step to
1e-13; the FP64 GPU path too, the mixed path to its default (2e-7)."""
import numpy as np
import pytest

import oracle as O
from paper_1808_04099_gb300 import workloads as W
from _util import assert_close, demean_per_sim, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1808_04099_gb300 import bcm  # noqa: E402

TOL64, TOL32 = 1e-10, 1e-6

def two_level_with_bodies():
    """The two-level channel with a fixed sphere and a moving ellipsoid inside the
    refined block (without bodies its pressure is ~1e-4 of the velocity, too small for a
    relative comparison of an FP32 state: rounding the state alone moves it by 1e-4)."""
    spec = W.two_level_channel(4, 4, 4, 8, (1, 1, 1), (3, 3, 3), 1 / 16., 0)
    q = np.array([0.9, 0.1, 0.3, 0.3])
    spec.bodies = [[W.Body(W.BODY_SPHERE, np.array([0.9, 1.0, 1.0]), np.array([0.22] * 3)),
                    W.Body(W.BODY_ELLIPSOID, np.array([1.25, 0.9, 1.1]),
                           np.array([0.12, 0.07, 0.09]), q / np.linalg.norm(q),
                           np.array([0.4, -1.0, 0.6]), np.array([0.02, 0.0, 0.0]))]]
    return spec


GRIDS = {
    "sphere_B8": lambda: W.sphere_channel(4, 2, 2, 8, radius=0.3),
    "cavity_B8": lambda: W.cavity(2, 8, re=400.0),
    "periodic_B4": lambda: W.periodic_box(2, 4),
    "sphere_B16": lambda: W.sphere_channel(2, 1, 1, 16, length=(2.0, 1.0, 1.0), radius=0.2,
                                           center=(0.6, 0.5, 0.5)),
    "two_level": lambda: W.two_level_channel(4, 4, 4, 8, (1, 1, 1), (3, 3, 3), 1 / 16., 0),
    "two_level_bodies": two_level_with_bodies,
    "batched": lambda: W.concat([W.cavity(2, 4, re=300.0), W.sphere_channel(4, 2, 2, 4, radius=0.3),
                                 W.periodic_box(2, 4)]),
}


def oracle_cn(spec, state, steps, schemes=None):
    o = O.Oracle(spec)
    st = o.new_state(state)
    stats = None
    for sch in (schemes or [1] * steps):
        o.set_scheme(sch, 1e-13, 500)
        stats, rc = o.step(st, 1, rtol=1e-13)
        assert rc == 0
    return st, stats


def velocity(g):
    return np.concatenate([g.numpy(f) for f in (bcm.U, bcm.V, bcm.W)])


def compare(g, ost, spec, tol):
    ref = np.concatenate([ost[k] for k in ("u", "v", "w")])
    assert_close(velocity(g), ref, g.numpy(bcm.P), ost["p"], spec, tol)


def gpu_cn(spec, state, prec, cn_rtol=None):
    g = bcm.Grid(spec, prec)
    g.load_state(state)
    g.set_momentum_scheme(bcm.SCHEME_QUICK_CN, 1e-13 if cn_rtol is None and prec == bcm.PREC_F64
                          else (cn_rtol or 0.0), 500)
    return g


@pytest.mark.parametrize("name", sorted(GRIDS))
def test_cn_steps_fp64_match_oracle(name):
    spec = GRIDS[name]()
    state = W.initial_state(spec, seed=41, noise=1e-3)
    ost, ostats = oracle_cn(spec, state, 3)
    g = gpu_cn(spec, state, bcm.PREC_F64)
    st = g.step(3, rtol=1e-13)
    assert all(s["converged"] == 1 for s in st)
    compare(g, ost, spec, TOL64)
    for s, o in zip(st, ostats):
        assert np.allclose(s["drag"], o["drag"], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("name", ["sphere_B8", "sphere_B16", "two_level_bodies", "batched"])
def test_cn_steps_mixed_match_oracle(name):
    spec = GRIDS[name]()
    state = W.initial_state(spec, seed=42, noise=1e-3)
    ost, _ = oracle_cn(spec, state, 3)
    g = gpu_cn(spec, state, bcm.PREC_F32_REFINE)
    st = g.step(3, rtol=1e-12)
    assert all(s["converged"] == 1 for s in st)
    compare(g, ost, spec, TOL32)


def test_cn_graph_steps_match_oracle():
    spec = GRIDS["sphere_B8"]()
    state = W.initial_state(spec, seed=43, noise=1e-3)
    ost, _ = oracle_cn(spec, state, 3)
    g = gpu_cn(spec, state, bcm.PREC_F32_REFINE)
    g.step_graph(3, rtol=1e-12)
    compare(g, ost, spec, TOL32)


def test_switch_back_to_adams_bashforth():
    spec = GRIDS["sphere_B8"]()
    state = W.initial_state(spec, seed=44, noise=1e-3)
    ost, _ = oracle_cn(spec, state, 3, schemes=[0, 1, 0])
    g = bcm.Grid(spec, bcm.PREC_F64)
    g.load_state(state)
    g.step(1, rtol=1e-13)
    g.set_momentum_scheme(bcm.SCHEME_QUICK_CN, 1e-13, 500)
    g.step(1, rtol=1e-13)
    g.set_momentum_scheme(bcm.SCHEME_AB2_CENTRAL)
    g.step(1, rtol=1e-13)
    compare(g, ost, spec, TOL64)


def test_cn_with_lagrangian_particles():
    spec = W.sphere_channel(4, 2, 2, 8, length=(2.0, 1.0, 1.0), radius=0.2,
                            center=(0.8, 0.5, 0.45))
    parts = W.surface_particles(spec, seed=45)
    state = W.initial_state(spec, seed=46, noise=1e-3)
    o = O.Oracle(spec)
    o.set_scheme(1, 1e-13, 500)
    ost = o.new_state(state)
    X = parts.X.copy()
    ostats, rc, _ = o.step_particles(ost, X, parts, nsteps=2, rtol=1e-13)
    assert rc == 0
    g = gpu_cn(spec, state, bcm.PREC_F64)
    g.set_particles(parts)
    st = g.step(2, rtol=1e-13)
    compare(g, ost, spec, TOL64)
    assert np.allclose(st[0]["drag"], ostats[0]["drag"], rtol=1e-9, atol=1e-12)


def test_scheme_rejects_bad_arguments():
    g = bcm.Grid(GRIDS["cavity_B8"](), bcm.PREC_F64)
    for args in ((7, 0.0, 0), (1, -1.0, 0), (1, 0.0, -2)):
        with pytest.raises(bcm.BCMError) as ei:
            g.set_momentum_scheme(*args)
        assert ei.value.status == bcm.BCM_E_INVALID


def test_full_size_sphere_cn_mixed():
    """The 4.19M-cell sphere flow, two steps with QUICK + Crank-Nicolson: mixed against
    FP64 on the GPU (1e-6)."""
    spec = W.config_sphere(2)
    state = W.initial_state(spec)
    out = []
    for prec in (bcm.PREC_F32_REFINE, bcm.PREC_F64):
        g = bcm.Grid(spec, prec)
        g.load_state(state)
        g.set_momentum_scheme(bcm.SCHEME_QUICK_CN)
        st = g.step(2, rtol=1e-10)
        assert st[0]["converged"] == 1
        out.append(velocity(g))
        del g
        torch.cuda.empty_cache()
    assert rel_l2(out[0], out[1]) <= TOL32
