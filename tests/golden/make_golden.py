"""Writes tests/golden/oracle_regression.json: what the oracle computes on small seeded
workloads, so that any later change to the oracle's arithmetic shows up as a mismatch
(tests/test_golden.py) and has to be regenerated on purpose.  It calls only oracle/
and the seeded input generators of paper_1808_04099_gb300/workloads.py.

    python tests/golden/make_golden.py

Each case names the passage of the paper its steps follow.  The paper prints no
worked example with numbers for any of them, so every stored value here comes from
the oracle itself."""
from __future__ import annotations

import json
import os
import sys
import zlib

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1808_04099_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "oracle_regression.json")


def _samples(f, k: int = 8):
    f = np.asarray(f, np.float64)
    idx = np.linspace(0, f.size - 1, k).astype(int)
    return {"index": idx.tolist(), "value": f[idx].tolist()}


def _digest(st):
    return {"norm": {k: float(np.linalg.norm(st[k])) for k in ("u", "v", "w", "p")},
            "samples": {k: _samples(st[k]) for k in ("u", "v", "w", "p")}}


def _steps(o, st, n, rtol):
    out = []
    for _ in range(n):
        stats, rc = o.step(st, 1, rtol=rtol)
        assert rc == 0
        s = stats[0]
        out.append({"cg_iters": int(s["cg_iters"]), "drag": [float(x) for x in s["drag"]],
                    "div_rel": float(s["div_rel"]), "umax": float(s["umax"])})
    return out


def case_step(spec, seed, noise, n, rtol=1e-12, scheme=None):
    o = O.Oracle(spec)
    if scheme is not None:
        o.set_scheme(*scheme)
    st = o.new_state(W.initial_state(spec, seed=seed, noise=noise))
    steps = _steps(o, st, n, rtol)
    return {"steps": steps, **_digest(st)}


def case_particles():
    spec = W.sphere_channel(4, 2, 2, 8, length=(2.0, 1.0, 1.0), radius=0.2,
                            center=(0.8, 0.5, 0.45))
    parts = W.surface_particles(spec, seed=72)
    o = O.Oracle(spec)
    st = o.new_state(W.initial_state(spec, seed=73, noise=1e-3))
    X = parts.X.copy()
    stats, rc, F = o.step_particles(st, X, parts, nsteps=2, rtol=1e-12)
    assert rc == 0
    return {"particles": int(parts.n), "drag": [float(x) for x in stats[0]["drag"]],
            "force_norm": float(np.linalg.norm(F)), **_digest(st)}


def case_wavelet():
    spec = W.sphere_channel(4, 2, 2, 8, radius=0.3)
    o = O.Oracle(spec)
    st = o.new_state(W.initial_state(spec, seed=2, noise=1e-3))
    _steps(o, st, 1, 1e-12)
    out = {}
    for key in ("u", "p"):
        f = st[key]
        step = 1e-4 * float(np.abs(f).max())
        words = O.wavelet_compress(f, spec.B, step)
        back = O.wavelet_decompress(words)
        out[key] = {"step": step, "words": int(words.size),
                    "crc32": int(zlib.crc32(np.ascontiguousarray(words, np.uint32).tobytes())),
                    "max_error_over_step": float(np.abs(back - f).max() / step)}
    return out


CASES = {
    "cavity_2x2x2_B4": (
        'Section "Numerical algorithm" (Eq. substep1, Eq. poisson, the projection); '
        'no-slip walls and a moving lid',
        lambda: case_step(W.cavity(2, 4), 1, 1e-2, 3)),
    "sphere_channel_4x2x2_B8": (
        'Section "Numerical algorithm" with the constraint forcing of section '
        '"Lagrangian--Eulerian approach" read as a solid fraction (R5 of the oracle); '
        'inflow, convective outflow, slip',
        lambda: case_step(W.sphere_channel(4, 2, 2, 8, radius=0.3), 2, 1e-3, 2)),
    "two_level_4x2x2_B4": (
        'Section "Building Cube Method" (halo rules across 2:1 faces) with the step of '
        'section "Numerical algorithm"',
        lambda: case_step(W.two_level_channel(4, 2, 2, 4, (1, 0, 0), (3, 2, 2), 1 / 8., 0),
                          4, 1e-3, 2)),
    "periodic_2x2x2_B4": (
        'Section "Numerical algorithm" on an all-periodic box (all-Neumann pressure gauge)',
        lambda: case_step(W.periodic_box(2, 4), 5, 1e-1, 2)),
    "quick_cn_sphere_channel_4x2x2_B8": (
        'Section "Numerical algorithm": QUICK convection with Crank-Nicolson (Eq. substep1)',
        lambda: case_step(W.sphere_channel(4, 2, 2, 8, radius=0.3), 2, 1e-3, 2,
                          scheme=(1, 1e-13, 500))),
    "particles_sphere_channel_4x2x2_B8": (
        'Section "Lagrangian-Eulerian Interaction": particles with the 3-point delta '
        '(Eq. ddeltai, Eq. ddeltap)',
        case_particles),
    "wavelet_sphere_channel_4x2x2_B8": (
        'Section "Data compression": per-cube wavelet transform, one quantizer, '
        'entropy coding (the Rice coder of the oracle stands in for zlib)',
        case_wavelet),
}


def compute() -> dict:
    return {name: {"cite": cite, "values": fn()} for name, (cite, fn) in CASES.items()}


if __name__ == "__main__":
    data = {"generator": "tests/golden/make_golden.py (calls only oracle/ and the seeded "
                         "input generators)",
            "cases": compute()}
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1)
    print(f"wrote {OUT}")
