"""Launch-shape autotuner of the PCG: the persistent cooperative solver (two passes per
iteration streaming with 1, 2 or 4 z-slabs per work item or with the search direction
in shared memory, the fused single-barrier form with bulk-copy staging, or the
single-reduction form), or two launches per iteration with z-slabs per pass.

Times a fixed number of PCG iterations on the grid's current right-hand side for
every shape with the library's own CUDA-event kernel timing, restores the pressure,
and keeps the fastest shape.  Results are cached in a JSON file keyed by device,
cube size, precision and cube count.
"""
from __future__ import annotations

import json
import os

from . import bcm

# (persistent, slabs_a, slabs_b)
SHAPES = [(5, 1, 1), (1, 1, 1), (1, 2, 1), (1, 4, 1), (3, 1, 1), (2, 1, 1), (2, 2, 1),
          (2, 4, 1), (0, 1, 1), (0, 1, 2), (0, 2, 2)]
CACHE = os.path.join(os.path.expanduser("~"), ".cache", "bcm_gb300_launch.json")


def _key(grid, device_name=None) -> str:
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name(grid.device)
    # the shape list is part of the key: a cache written for other shapes is not used
    shapes = ";".join(f"{pe},{sa},{sb}" for pe, sa, sb in SHAPES)
    return (f"{device_name}|B{grid.spec.B}|prec{grid.precision}|cubes{grid.spec.n_cubes}"
            f"|shapes{shapes}")


def _read_cache(path: str) -> dict:
    try:
        with open(path) as f:
            cache = json.load(f)
        return cache if isinstance(cache, dict) else {}
    except (OSError, ValueError):
        return {}


def tune(grid, iters: int = 40, use_cache: bool = True, cache_path: str | None = None,
         device_name: str | None = None) -> dict:
    """Pick and set the fastest launch shape; returns {"persistent,slabs_a,slabs_b": us
    per iteration}.  The cache (a JSON file, cache_path or CACHE) maps the device, cube
    size, precision, cube count and shape list to the best shape and its times; an
    unreadable cache counts as empty.  The caller's solver controls are restored."""
    path = cache_path or CACHE
    key = _key(grid, device_name) if use_cache else None
    cache = _read_cache(path) if use_cache else {}
    entry = cache.get(key)
    if use_cache and isinstance(entry, dict) and tuple(entry.get("best", ())) in SHAPES:
        pe, sa, sb = entry["best"]
        grid.set_launch(sa, sb, persistent=pe)
        return entry["times"]
    p = grid.field(bcm.P)
    saved = p.clone()
    times = {}
    caller_cycles = grid.get_solver()["max_cycles"]
    grid.set_solver(max_cycles=1)  # mixed mode: one inner solve per timing run
    try:
        _time_shapes(grid, iters, p, saved, times)
    finally:
        p.copy_(saved)
        grid.set_solver(max_cycles=caller_cycles)
    best = min(times, key=times.get)
    pe, sa, sb = map(int, best.split(","))
    grid.set_launch(sa, sb, persistent=pe)
    if use_cache:
        cache = _read_cache(path)  # another process may have added entries meanwhile
        cache[key] = {"best": [pe, sa, sb], "times": times}
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    return times


def _time_shapes(grid, iters, p, saved, times):
    """us per PCG iteration of every launch shape, into times.  Each includes its share
    of the defect correction's x += e (one per inner solve): the streaming form does it
    at the end of its own launch, the others in a launch of their own."""
    for pe, sa, sb in SHAPES:
        if pe and sa > 1 and grid.spec.B != 16:
            continue
        if pe == 5 and (grid.spec.B != 16 or grid.precision == bcm.PREC_F64):
            continue  # the fused form runs FP32 inner solves on 16^3 cubes only
        grid.set_launch(sa, sb, persistent=pe)
        for rep in range(2):  # the first pass warms up the shape
            p.copy_(saved)
            grid.profile(True)
            grid.solve_pressure_iters(iters)
            prof, _ = grid.profile_read(reset=True)
            grid.profile(False)
        ta, na = prof["cg_a"]
        tb, nb = prof["cg_b"]
        tp, npc = prof["pcg"]
        tc, nc = prof.get("add_correction", (0.0, 0))
        corr = tc / (nc * iters) if nc else 0.0
        if pe and npc:
            times[f"{pe},{sa},{sb}"] = 1e3 * (tp / (npc * iters) + corr)
        elif na and nb:
            times[f"{pe},{sa},{sb}"] = 1e3 * (ta / na + tb / nb + corr)


STENCIL_SLABS = (1, 2, 4)
STATE_FIELDS = (bcm.U, bcm.V, bcm.W, bcm.P, bcm.NX, bcm.NY, bcm.NZ, bcm.UB)


def tune_stencils(grid, steps: int = 2, use_cache: bool = True, cache_path: str | None = None,
                  device_name: str | None = None) -> dict:
    """Pick and set the fastest z-slab depth of the momentum and right-hand-side kernels
    on 16^3 cubes (bcm_set_stencil_slabs); returns {slabs: us per step of the two}.  Each
    depth is timed over `steps` steps with the library's kernel timing after one warm-up
    step; the state, the time and the caller's setting are restored afterwards (the
    running drag mean of bcm_drag_mean counts the timing steps).  Cached like tune()."""
    if grid.spec.B != 16:
        return {}
    path = cache_path or CACHE
    key = None
    if use_cache:
        key = "stencil|" + _key(grid, device_name) + "|slabs" + ",".join(map(str, STENCIL_SLABS))
        entry = _read_cache(path).get(key)
        if isinstance(entry, dict) and entry.get("best") in STENCIL_SLABS:
            grid.set_stencil_slabs(entry["best"])
            return {int(k): v for k, v in entry["times"].items()}
    saved = [grid.field(f).clone() for f in STATE_FIELDS]
    step0 = grid.step(0)[0]["steps"]
    caller = grid.get_stencil_slabs()
    times = {}
    try:
        for ns in STENCIL_SLABS:
            grid.set_stencil_slabs(ns)
            for rep in range(2):  # a warm-up step, then the timed steps
                for f, t in zip(STATE_FIELDS, saved):
                    grid.field(f).copy_(t)
                grid.set_step(step0)
                grid.profile(True)
                grid.step(1 if rep == 0 else steps, stats=False)
                prof, _ = grid.profile_read(reset=True)
                grid.profile(False)
            tm, nm = prof["momentum"]
            tr, nr = prof["rhs"]
            if nm and nr:
                times[ns] = 1e3 * (tm / nm + tr / nr)
    finally:
        for f, t in zip(STATE_FIELDS, saved):
            grid.field(f).copy_(t)
        grid.set_step(step0)
        grid.set_stencil_slabs(caller)
    if not times:
        return times
    best = min(times, key=times.get)
    grid.set_stencil_slabs(best)
    if use_cache:
        cache = _read_cache(path)
        cache[key] = {"best": best, "times": {str(k): v for k, v in times.items()}}
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    return times
