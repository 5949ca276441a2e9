"""CUDA-graph-captured steps (bcm_step_graph) against the FP64 oracle and against the
eagerly issued steps: the captured step has no host synchronisation, runs the
persistent PCG and a fixed budget of defect-correction cycles."""
import numpy as np
import pytest

from paper_1808_04099_gb300 import workloads as W
from _util import assert_close, demean_per_sim, oracle_run, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1808_04099_gb300 import bcm  # noqa: E402

TOL64, TOL32 = 1e-10, 1e-6


def velocity(g):
    return np.concatenate([g.numpy(f) for f in (bcm.U, bcm.V, bcm.W)])


def check(g, ost, spec, tol):
    ref = np.concatenate([ost[k] for k in ("u", "v", "w")])
    assert_close(velocity(g), ref, g.numpy(bcm.P), ost["p"], spec, tol)


@pytest.mark.parametrize("prec", [bcm.PREC_F64, bcm.PREC_F32_REFINE])
def test_graph_steps_match_oracle_and_eager(prec):
    spec = W.sphere_channel(4, 2, 2, 8, radius=0.3)
    state = W.initial_state(spec, seed=41)
    ost, ostats = oracle_run(spec, state, 3, 1e-13)
    rtol = 1e-13 if prec == bcm.PREC_F64 else 1e-12
    tol = TOL64 if prec == bcm.PREC_F64 else TOL32
    g = bcm.Grid(spec, prec)
    g.load_state(state)
    st = g.step_graph(1, rtol=rtol)           # captures, then replays
    st = g.step_graph(2, rtol=rtol)           # replays the same graph
    assert st[0]["steps"] == 3 and st[0]["converged"] == 1
    check(g, ost, spec, tol)
    e = bcm.Grid(spec, prec)
    e.load_state(state)
    e.set_launch(1, 1, persistent=True)
    e.step(3, rtol=rtol)
    assert rel_l2(velocity(g), velocity(e)) <= tol
    assert abs(st[0]["drag"][0] - ostats[0]["drag"][0]) <= 1e-6 * abs(ostats[0]["drag"][0])


@pytest.mark.parametrize("prec", [bcm.PREC_F64, bcm.PREC_F32_REFINE])
def test_graph_single_pass_pcg(prec):
    """The captured step with the single-reduction persistent PCG."""
    spec = W.sphere_channel(4, 2, 2, 8, radius=0.3)
    state = W.initial_state(spec, seed=44)
    ost, _ = oracle_run(spec, state, 3, 1e-13)
    g = bcm.Grid(spec, prec)
    g.load_state(state)
    g.set_launch(1, 1, persistent=2)
    st = g.step_graph(3, rtol=1e-13 if prec == bcm.PREC_F64 else 1e-12)
    assert st[0]["converged"] == 1
    check(g, ost, spec, TOL64 if prec == bcm.PREC_F64 else TOL32)


def test_graph_batched_sims():
    """Independent cavity and sphere sims of uneven size in one captured step."""
    specs = [W.cavity(2, 8, re=250.0), W.sphere_channel(4, 2, 2, 8, radius=0.3, re=500.0),
             W.cavity(3, 8, re=800.0)]
    spec = W.concat(specs)
    state = W.initial_state(spec, seed=42, noise=1e-3)
    ost, _ = oracle_run(spec, state, 3, 1e-13)
    g = bcm.Grid(spec, bcm.PREC_F32_REFINE)
    g.load_state(state)
    st = g.step_graph(3, rtol=1e-12)
    assert all(s["converged"] == 1 for s in st)
    check(g, ost, spec, TOL32)


def test_graph_moving_bodies_two_level():
    """Moving bodies re-evaluate their solid fraction inside the graph from the device
    step counter, on a two-level grid."""
    spec = W.two_level_channel(4, 4, 4, 8, (1, 1, 1), (3, 3, 3), 1 / 16., 0)
    spec.bodies = [[W.Body(W.BODY_ELLIPSOID, np.array([1.0, 1.0, 1.0]),
                           np.array([0.2, 0.1, 0.15]), np.array([1.0, 0, 0, 0]),
                           np.array([0.0, 0.8, 0.3]), np.array([0.05, 0.0, 0.0]))]]
    state = W.initial_state(spec, seed=43)
    ost, _ = oracle_run(spec, state, 3, 1e-13)
    g = bcm.Grid(spec, bcm.PREC_F64)
    g.load_state(state)
    g.step_graph(3, rtol=1e-13)
    check(g, ost, spec, TOL64)
