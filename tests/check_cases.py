"""Small steps on every staged-tile path, written to an .npz: run once with the default
library and once with the checked build (BCM_CHECK=1 in the environment selects
libbcm_check.so) by tests/test_gpu_check.py, which compares the two.

    python tests/check_cases.py OUT.npz
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1808_04099_gb300 import bcm  # noqa: E402
from paper_1808_04099_gb300 import workloads as W  # noqa: E402


def two_level():
    return W.two_level_channel(4, 2, 2, 8, (1, 0, 0), (3, 2, 2), 1 / 16., 1, seed=3)


# name: (spec, precision, launch (persistent, slabs_a, slabs_b) or None, preconditioner,
#        momentum scheme, graph steps, steps)
CASES = {
    "sphere_mixed_streaming": (lambda: W.sphere_channel(4, 2, 2, 8, radius=0.3),
                               bcm.PREC_F32_REFINE, (1, 1, 1), bcm.PRECOND_JACOBI,
                               bcm.SCHEME_AB2_CENTRAL, False, 2),
    "two_level_fp64": (two_level, bcm.PREC_F64, None, bcm.PRECOND_JACOBI,
                       bcm.SCHEME_AB2_CENTRAL, False, 2),
    "two_level_mixed_multigrid": (two_level, bcm.PREC_F32_REFINE, None,
                                  bcm.PRECOND_MULTIGRID, bcm.SCHEME_AB2_CENTRAL, False, 2),
    "cavity16_graph": (lambda: W.cavity(2, 16), bcm.PREC_F32_REFINE, (1, 2, 1),
                       bcm.PRECOND_JACOBI, bcm.SCHEME_AB2_CENTRAL, True, 2),
    "sphere_quick_cn": (lambda: W.sphere_channel(4, 2, 2, 8, radius=0.3), bcm.PREC_F64, None,
                        bcm.PRECOND_JACOBI, bcm.SCHEME_QUICK_CN, False, 1),
    "periodic_two_launch": (lambda: W.periodic_box(2, 8), bcm.PREC_F64, (0, 2, 2),
                            bcm.PRECOND_JACOBI, bcm.SCHEME_AB2_CENTRAL, False, 2),
}


def main(out):
    res = {}
    for name, (mk, prec, launch, pre, scheme, graph, steps) in CASES.items():
        spec = mk()
        g = bcm.Grid(spec, prec)
        g.load_state(W.initial_state(spec, seed=61, noise=1e-3))
        if launch is not None:
            pe, sa, sb = launch
            g.set_launch(sa, sb, persistent=pe)
        g.set_preconditioner(pre)
        g.set_momentum_scheme(scheme)
        rtol = 1e-12 if prec == bcm.PREC_F64 else 1e-10
        st = g.step_graph(steps, rtol=rtol) if graph else g.step(steps, rtol=rtol)
        assert all(s["converged"] == 1 for s in st), (name, st)
        res[name] = np.concatenate([g.numpy(f) for f in (bcm.U, bcm.V, bcm.W, bcm.P)])
        del g
    np.savez(out, **res)
    print("cases", len(res), "library", bcm.lib()._name)


if __name__ == "__main__":
    main(sys.argv[1])
