"""Options of the library used together, against the oracle: the multigrid
preconditioner under QUICK + Crank-Nicolson momentum and under the particle IB (the
pressure solution is unique, so the oracle's Jacobi PCG gives the same fields), and
wavelet compression of a two-level grid's fields (per cube, whatever its level)."""
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


def velocity(g):
    return np.concatenate([g.numpy(f) for f in (bcm.U, bcm.V, bcm.W)])


def compare(g, ost, spec, tol):
    ref = np.concatenate([ost[k] for k in ("u", "v", "w")])
    assert_close(velocity(g), ref, g.numpy(bcm.P), ost["p"], spec, tol)


@pytest.mark.parametrize("prec", [bcm.PREC_F64, bcm.PREC_F32_REFINE])
def test_multigrid_with_crank_nicolson(prec):
    spec = W.sphere_channel(4, 2, 2, 8, radius=0.3)
    state = W.initial_state(spec, seed=71, noise=1e-3)
    o = O.Oracle(spec)
    o.set_scheme(1, 1e-13, 500)
    ost = o.new_state(state)
    _, rc = o.step(ost, 2, rtol=1e-13)
    assert rc == 0
    g = bcm.Grid(spec, prec)
    g.load_state(state)
    g.set_preconditioner(bcm.PRECOND_MULTIGRID)
    g.set_momentum_scheme(bcm.SCHEME_QUICK_CN, 1e-13 if prec == bcm.PREC_F64 else 0.0, 500)
    st = g.step(2, rtol=1e-13 if prec == bcm.PREC_F64 else 1e-12)
    assert st[0]["converged"] == 1 and st[0]["pcg_form"] == 4 and st[0]["cn_iters"] > 0
    compare(g, ost, spec, 1e-10 if prec == bcm.PREC_F64 else 1e-6)


def test_multigrid_with_particles():
    spec = W.sphere_channel(4, 2, 2, 8, length=(2.0, 1.0, 1.0), radius=0.2,
                            center=(0.8, 0.5, 0.45))
    parts = W.surface_particles(spec, seed=72)
    state = W.initial_state(spec, seed=73, noise=1e-3)
    o = O.Oracle(spec)
    ost = o.new_state(state)
    X = parts.X.copy()
    ostats, rc, _ = o.step_particles(ost, X, parts, nsteps=2, rtol=1e-13)
    assert rc == 0
    g = bcm.Grid(spec, bcm.PREC_F64)
    g.load_state(state)
    g.set_preconditioner(bcm.PRECOND_MULTIGRID)
    g.set_particles(parts)
    st = g.step(2, rtol=1e-13)
    assert st[0]["pcg_form"] == 4
    compare(g, ost, spec, 1e-10)
    assert np.allclose(st[0]["drag"], ostats[0]["drag"], rtol=1e-9, atol=1e-12)


def test_wavelet_streams_of_a_two_level_grid():
    spec = W.two_level_channel(4, 4, 4, 8, (1, 1, 1), (3, 3, 3), 1 / 16., 0)
    g = bcm.Grid(spec, bcm.PREC_F32_REFINE)
    g.load_state(W.initial_state(spec, seed=74, noise=1e-2))
    g.step(1, rtol=1e-10)
    for fid in (bcm.U, bcm.P):
        f = g.numpy(fid)
        step = 1e-4 * np.abs(f).max()
        s = g.compress_field(fid, step).cpu().numpy().view(np.uint32)
        assert np.array_equal(s, O.wavelet_compress(f, spec.B, step))
