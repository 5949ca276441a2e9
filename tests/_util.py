"""Shared test helpers: run the oracle and the CUDA path on the same seeded inputs."""
import numpy as np

import oracle as O
from paper_1808_04099_gb300 import workloads as W


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def demean_per_sim(p, spec):
    """Pressure up to a constant in all-Neumann sims: remove each such sim's mean."""
    p = np.array(p, np.float64, copy=True)
    B3 = spec.B ** 3
    for s in range(spec.n_sims):
        if W.OUTFLOW in list(spec.sim_bc[s]):
            continue
        a, b = spec.sim_cube_offset[s] * B3, spec.sim_cube_offset[s + 1] * B3
        p[a:b] -= p[a:b].mean()
    return p


def oracle_run(spec, state, steps, rtol):
    o = O.Oracle(spec)
    st = o.new_state(state)
    stats, rc = o.step(st, steps, rtol=rtol)
    assert rc == 0
    return st, stats
