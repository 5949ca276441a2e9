"""The streaming PCG applies an iteration's x += alpha p while the next iteration
stages p, and the last one at the end of its launch; the two-launch form updates x in
its second pass.  After exactly k iterations (k = 1, 2, 3, 7) both hold the same
iterate up to rounding, for a sim whose zero right-hand side stops it before its
first iteration beside one that runs: in FP64, and in the FP32 inner solve of one
defect-correction cycle (where the streaming launch also adds e to the FP64
iterate)."""
import numpy as np
import pytest

from paper_1808_04099_gb300 import workloads as W
from _util import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1808_04099_gb300 import bcm  # noqa: E402

STREAMING, TWO_LAUNCH = 1, 0


def two_sims():
    return W.concat([W.sphere_channel(2, 1, 1, 16, length=(2.0, 1.0, 1.0), radius=0.2,
                                      center=(0.6, 0.5, 0.5)),
                     W.sphere_channel(2, 2, 1, 16, length=(2.0, 2.0, 1.0), radius=0.3,
                                      center=(1.0, 1.0, 0.5))])


def run(spec, prec, form, k, rhs):
    g = bcm.Grid(spec, prec)
    g.load_state(W.initial_state(spec, seed=5, noise=1e-3))
    g.set_launch(1, 1, persistent=form)
    g.set_solver(inner_rtol=1e-30, max_cycles=1)  # exactly k inner iterations, one cycle
    g.field(bcm.RHS).copy_(torch.from_numpy(rhs).to(g.field(bcm.RHS)))
    g.field(bcm.P).zero_()
    st = g.solve_pressure_iters(k)
    return g.numpy(bcm.P), st


@pytest.mark.parametrize("prec,tol", [(bcm.PREC_F64, 1e-12), (bcm.PREC_F32_REFINE, 1e-5)])
def test_iterate_after_exactly_k_iterations(prec, tol):
    spec = two_sims()
    B3 = spec.B ** 3
    cut = int(spec.sim_cube_offset[1]) * B3  # sim 0's cells
    rhs = np.random.default_rng(17).standard_normal(spec.n_cells)
    rhs[:cut] = 0.0
    for k in (1, 2, 3, 7):
        ps, sts = run(spec, prec, STREAMING, k, rhs)
        pt, stt = run(spec, prec, TWO_LAUNCH, k, rhs)
        assert sts[1]["pcg_form"] == STREAMING and stt[1]["pcg_form"] == TWO_LAUNCH
        assert sts[1]["cg_iters"] == stt[1]["cg_iters"] == k
        assert np.all(ps[:cut] == 0.0) and np.all(pt[:cut] == 0.0)
        # the last iteration's update is in: without it the iterates differ by alpha p
        assert rel_l2(ps[cut:], pt[cut:]) <= tol, (k, rel_l2(ps[cut:], pt[cut:]))
