"""Shared test helpers: run the oracle and the CUDA path on the same seeded inputs."""
import numpy as np

import oracle as O
from paper_1808_04099_gb300 import workloads as W


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def max_rel(a, b):
    """Largest cell error against the largest reference value: an error confined to a
    few cells (a face, the 2:1 interface, the body shell) shows here even when the
    relative L2 norm over millions of cells hides it."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


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


MAX_FACTOR = 10.0  # per-cell bound: max |a - b| <= MAX_FACTOR * tol * max |b|


def assert_close(vel, ref_vel, p, ref_p, spec, tol):
    """Velocity (as one vector) and pressure (mean removed in all-Neumann sims) within
    tol in relative L2, and every cell within MAX_FACTOR * tol of the largest value."""
    pg, pr = demean_per_sim(p, spec), demean_per_sim(ref_p, spec)
    ev, ep = rel_l2(vel, ref_vel), rel_l2(pg, pr)
    mv, mp = max_rel(vel, ref_vel), max_rel(pg, pr)
    assert ev <= tol and ep <= tol, ("relative L2", ev, ep, tol)
    assert mv <= MAX_FACTOR * tol and mp <= MAX_FACTOR * tol, ("largest cell", mv, mp, tol)
    return ev, ep, mv, mp


def oracle_run(spec, state, steps, rtol):
    o = O.Oracle(spec)
    st = o.new_state(state)
    stats, rc = o.step(st, steps, rtol=rtol)
    assert rc == 0
    return st, stats
