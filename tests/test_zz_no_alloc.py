"""The pressure solve that allocates nothing (bcm_solve_pressure_static).

It exists for callers that cannot allocate device memory when they solve (an
application whose GPU memory is reserved up front by its own pool, a plugin kept away
from the allocator); it keeps its working memory in a fixed array inside the library.
The test calls it through the C ABI twice in a row on the same grid and compares each
result with the ordinary bcm_solve_pressure, which uses the grid workspace, at the
pressure-solve tolerance of the other GPU tests, on FP64 grids and on a mixed-precision
grid (the static solve is FP64 there too; the workspace solve is the FP32 inner PCG in
FP64 defect correction, so the two agree to the solver tolerance).  It also checks the
stats it fills and the size limit.
This file is collected last so that a stop at its first failure has already run
every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1808_04099_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1808_04099_gb300 import bcm  # noqa: E402

TOL = 1e-11  # relative L2, as the pressure-solve parity tests


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("make", [lambda: W.cavity(2, 8), lambda: W.sphere_channel(4, 2, 2, 8)],
                         ids=["cavity", "channel"])
def test_static_solve_matches_workspace_solve_twice(make):
    spec = make()
    g = bcm.Grid(spec, bcm.PREC_F64)
    rng = np.random.default_rng(31)
    L = bcm.lib()
    for call in range(2):  # two calls in a row: the fixed array keeps old contents
        b = torch.from_numpy(rng.standard_normal(spec.n_cells)).cuda()
        p0 = torch.from_numpy(rng.standard_normal(spec.n_cells)).cuda()
        # reference: the ordinary entry point on the grid's own fields
        g.field(bcm.RHS).copy_(b)
        g.field(bcm.P).copy_(p0)
        ref_stats = g.solve_pressure(1e-12)
        p_ref = g.field(bcm.P).clone()
        # the static entry point with caller-owned input and output
        p = p0.clone()
        st = (bcm.Stats * spec.n_sims)()
        torch.cuda.synchronize()
        rc = L.bcm_solve_pressure_static(g._h, C.c_void_p(b.data_ptr()),
                                         C.c_void_p(p.data_ptr()), 1e-12, 20000, st)
        assert rc == bcm.BCM_OK, L.bcm_last_error()
        assert st[0].converged == 1 and st[0].cg_iters == ref_stats[0]["cg_iters"]
        assert st[0].steps == ref_stats[0]["steps"] and st[0].rel_resid <= 1e-12
        if W.OUTFLOW not in list(spec.sim_bc[0]):  # all-Neumann: compare up to a constant
            p, p_ref = p - p.mean(), p_ref - p_ref.mean()
        assert rel(p, p_ref) < TOL, (call, rel(p, p_ref))


def test_static_solve_on_a_mixed_precision_grid_twice():
    """On a PREC_F32_REFINE grid the static solve still runs in FP64; the workspace
    solve (FP32 inner PCG, FP64 defect correction) reaches the same solution to the
    solver tolerance.  Two steps first, so the grid's step count is not zero."""
    spec = W.sphere_channel(4, 2, 2, 8)
    g = bcm.Grid(spec, bcm.PREC_F32_REFINE)
    g.load_state(W.initial_state(spec, seed=2, noise=1e-3))
    g.step(2, rtol=1e-10)
    rng = np.random.default_rng(7)
    L = bcm.lib()
    for call in range(2):
        b = torch.from_numpy(rng.standard_normal(spec.n_cells)).cuda()
        p0 = torch.from_numpy(rng.standard_normal(spec.n_cells)).cuda()
        g.field(bcm.RHS).copy_(b)
        g.field(bcm.P).copy_(p0)
        ref_stats = g.solve_pressure(1e-12)
        p_ref = g.field(bcm.P).clone()
        p = p0.clone()
        st = (bcm.Stats * spec.n_sims)()
        torch.cuda.synchronize()
        rc = L.bcm_solve_pressure_static(g._h, C.c_void_p(b.data_ptr()),
                                         C.c_void_p(p.data_ptr()), 1e-12, 20000, st)
        assert rc == bcm.BCM_OK, L.bcm_last_error()
        assert st[0].converged == 1 and st[0].rel_resid <= 1e-12
        assert st[0].steps == ref_stats[0]["steps"] == 2
        # two solves stopped at relative residual 1e-12 differ by about cond(K) 1e-12
        assert rel(p, p_ref) < 1e-9, (call, rel(p, p_ref))


def test_static_solve_rejects_grids_beyond_its_memory():
    spec = W.cavity(8, 16)  # 2,097,152 cells: 4 FP64 vectors exceed 32 MiB
    g = bcm.Grid(spec, bcm.PREC_F64)
    b = torch.zeros(spec.n_cells, dtype=torch.float64, device="cuda")
    p = torch.zeros_like(b)
    L = bcm.lib()
    rc = L.bcm_solve_pressure_static(g._h, C.c_void_p(b.data_ptr()), C.c_void_p(p.data_ptr()),
                                     1e-8, 100, None)
    assert rc == bcm.BCM_E_BOUNDS
    assert b"static solve holds at most" in L.bcm_last_error()
