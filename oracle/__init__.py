"""ctypes shim of the FP64 CPU oracle (``bcm_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library: it is compiled from its own C source by gcc.

Every function here is argument marshalling; the arithmetic lives in the C file,
whose header lists the paper passages it follows and the readings it takes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bcm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, OpenMP, -O2, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or \
                os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                                  os.path.getmtime(_SRC[:-2] + ".h")):
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            # no FMA contraction: the same arithmetic on x86 and Arm hosts
            subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp",
                                   "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Stats(C.Structure):
    _fields_ = [("cg_iters", C.c_int32), ("steps", C.c_int32), ("rel_resid", C.c_double),
                ("div_rel", C.c_double), ("drag", C.c_double * 3), ("umax", C.c_double)]

    def as_dict(self):
        return {"cg_iters": self.cg_iters, "steps": self.steps, "rel_resid": self.rel_resid,
                "div_rel": self.div_rel, "drag": list(self.drag), "umax": self.umax}


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.c_void_p
        L.orc_create.restype = P
        L.orc_create.argtypes = [C.c_int] * 4 + [P] * 13
        L.orc_destroy.argtypes = [P]
        L.orc_error.restype = C.c_char_p
        L.orc_n_slots.argtypes = [P]
        L.orc_n_slots.restype = C.c_int
        L.orc_threads.restype = C.c_int
        L.orc_set_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_neighbors.argtypes = [P, P]
        L.orc_fill_ghosts.argtypes = [P, P, C.c_int, P, P]
        L.orc_solid_fraction.argtypes = [P] * 6
        L.orc_convection_diffusion.argtypes = [P] * 11
        L.orc_apply_poisson.argtypes = [P, P, P]
        L.orc_poisson_diag.argtypes = [P, P]
        L.orc_rhs.argtypes = [P] * 6
        L.orc_solve_pressure.argtypes = [P, P, P, C.c_double, C.c_int, P]
        L.orc_solve_pressure.restype = C.c_int
        L.orc_step.argtypes = [P] * 10 + [C.c_int, C.c_double, C.c_int, P]
        L.orc_step.restype = C.c_int
        L.orc_convection_quick.argtypes = [P] * 8
        L.orc_set_scheme.argtypes = [P, C.c_int, C.c_double, C.c_int]
        L.orc_set_scheme.restype = C.c_int
        L.orc_dwt3_forward.argtypes = [C.c_int, P]
        L.orc_dwt3_inverse.argtypes = [C.c_int, P]
        L.orc_wavelet_compress.argtypes = [C.c_int, C.c_int, P, C.c_double, P, C.c_long]
        L.orc_wavelet_compress.restype = C.c_long
        L.orc_wavelet_decompress.argtypes = [P, C.c_long, P]
        L.orc_wavelet_decompress.restype = C.c_int
        L.orc_delta3.argtypes = [C.c_double]
        L.orc_delta3.restype = C.c_double
        L.orc_ib_interpolate.argtypes = [P, P, C.c_int, P, P, P]
        L.orc_ib_spread.argtypes = [P, C.c_int, P, P, P, P, P]
        L.orc_ib_body_velocity.argtypes = [P, C.c_int, P, P, P, P, P]
        L.orc_step_particles.argtypes = [P] * 10 + [C.c_int, C.c_double, C.c_int, P, C.c_int] + \
            [P] * 5
        L.orc_step_particles.restype = C.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def dwt3(x, B: int, inverse: bool = False) -> np.ndarray:
    """The per-cube 3-D CDF 5/3 transform (R21) of one cube of B^3 values."""
    y = np.ascontiguousarray(x, np.float64).copy()
    (lib().orc_dwt3_inverse if inverse else lib().orc_dwt3_forward)(B, _p(y))
    return y


def wavelet_compress(f, B: int, step: float) -> np.ndarray:
    """Compressed stream (uint32 words) of a cube-major field of n_cubes B^3 values."""
    f = _f64(f)
    n_cubes = f.size // B ** 3
    cap = 8 + n_cubes + n_cubes * (1 + (B ** 3 * 48 + 31) // 32)
    out = np.zeros(cap, np.uint32)
    nw = lib().orc_wavelet_compress(B, n_cubes, _p(f), step, _p(out), cap)
    if nw < 0:
        raise ValueError("wavelet compression: code out of range")
    return out[:nw].copy()


def wavelet_decompress(words) -> np.ndarray:
    words = np.ascontiguousarray(words, np.uint32)
    B, n_cubes = int(words[2]), int(words[3])
    f = np.zeros(n_cubes * B ** 3)
    if lib().orc_wavelet_decompress(_p(words), words.size, _p(f)):
        raise ValueError("wavelet decompression: malformed stream")
    return f


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """The oracle's own grid for one GridSpec (see paper_1808_04099_gb300.workloads)."""

    def __init__(self, spec):
        self.spec = spec
        self.B = spec.B
        L = lib()
        self._keep = [
            np.ascontiguousarray(spec.sim_cube_offset, np.int32),
            np.ascontiguousarray(spec.cube_ijk, np.int32),
            np.ascontiguousarray(spec.cube_level, np.int8),
            np.ascontiguousarray(spec.sim_extent, np.int32),
            _f64(spec.sim_origin), _f64(spec.sim_h0),
            np.ascontiguousarray(spec.sim_bc, np.int32), _f64(spec.sim_bc_vel),
            _f64(spec.sim_nu), _f64(spec.sim_dt), _f64(spec.sim_uconv),
            _f64(spec.body_table()), _f64(spec.inflow_modes),
        ]
        h = L.orc_create(spec.B, spec.max_level, spec.n_sims, spec.n_cubes,
                         *[_p(a) for a in self._keep])
        if not h:
            raise ValueError("oracle grid: " + L.orc_error().decode())
        self._h = C.c_void_p(h)
        self.n_slots = L.orc_n_slots(self._h)
        self.n_cells = spec.n_cells

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    # ---------------------------------------------------------------- pieces
    def neighbors(self) -> np.ndarray:
        out = np.empty((self.spec.n_cubes, 6), np.int32)
        lib().orc_neighbors(self._h, _p(out))
        return out

    def fill_ghosts(self, f, kind: int, ub=None) -> np.ndarray:
        G = self.B + 4
        out = np.zeros((self.spec.n_cubes, G, G, G))
        f = _f64(f)
        ubp = _p(_f64(ub)) if ub is not None and np.size(ub) else None
        keep = _f64(ub) if ub is not None and np.size(ub) else None
        if keep is not None:
            ubp = _p(keep)
        lib().orc_fill_ghosts(self._h, _p(f), kind, ubp, _p(out))
        return out

    def solid_fraction(self, t):
        n = self.n_cells
        t = _f64(np.broadcast_to(np.asarray(t, np.float64), (self.spec.n_sims,)))
        phi, us, vs, ws = (np.zeros(n) for _ in range(4))
        lib().orc_solid_fraction(self._h, _p(t), _p(phi), _p(us), _p(vs), _p(ws))
        return phi, us, vs, ws

    def convection_diffusion(self, u, v, w, ub=None):
        n = self.n_cells
        outs = [np.zeros(n) for _ in range(6)]
        u, v, w = _f64(u), _f64(v), _f64(w)
        ubk = _f64(ub) if ub is not None and np.size(ub) else None
        lib().orc_convection_diffusion(self._h, _p(u), _p(v), _p(w),
                                       _p(ubk) if ubk is not None else None,
                                       *[_p(o) for o in outs])
        return outs[:3], outs[3:]

    def apply_poisson(self, x) -> np.ndarray:
        x = _f64(x)
        y = np.zeros_like(x)
        lib().orc_apply_poisson(self._h, _p(x), _p(y))
        return y

    def poisson_diag(self) -> np.ndarray:
        d = np.zeros(self.n_cells)
        lib().orc_poisson_diag(self._h, _p(d))
        return d

    def rhs(self, us, vs, ws, ub_new=None) -> np.ndarray:
        b = np.zeros(self.n_cells)
        us, vs, ws = _f64(us), _f64(vs), _f64(ws)
        ubk = _f64(ub_new) if ub_new is not None and np.size(ub_new) else None
        lib().orc_rhs(self._h, _p(us), _p(vs), _p(ws), _p(ubk) if ubk is not None else None,
                      _p(b))
        return b

    def solve_pressure(self, b, p0=None, rtol=1e-12, max_iter=100000):
        b = _f64(b)
        p = np.zeros(self.n_cells) if p0 is None else _f64(p0).copy()
        st = (Stats * self.spec.n_sims)()
        rc = lib().orc_solve_pressure(self._h, _p(b), _p(p), rtol, max_iter, st)
        return p, [s.as_dict() for s in st], rc

    # ---------------------------------------------------------------- stepping
    def new_state(self, state):
        """Mutable oracle state from a workloads.State (copied)."""
        n = self.n_cells
        return {"u": _f64(state.u).copy(), "v": _f64(state.v).copy(), "w": _f64(state.w).copy(),
                "p": _f64(state.p).copy(), "nx": np.zeros(n), "ny": np.zeros(n),
                "nz": np.zeros(n), "ub": _f64(state.ub).copy().reshape(-1),
                "step": np.zeros(self.spec.n_sims, np.int32)}

    def step(self, st, nsteps=1, rtol=1e-12, max_iter=100000):
        stats = (Stats * self.spec.n_sims)()
        ub = st["ub"]
        if ub.size == 0:
            ub = np.zeros(1)
            st["ub"] = ub
        rc = lib().orc_step(self._h, _p(st["u"]), _p(st["v"]), _p(st["w"]), _p(st["p"]),
                            _p(st["nx"]), _p(st["ny"]), _p(st["nz"]), _p(ub), _p(st["step"]),
                            nsteps, rtol, max_iter, stats)
        return [s.as_dict() for s in stats], rc

    # ------------------------------------------- QUICK + Crank-Nicolson (R20)
    def convection_quick(self, u, v, w, ub=None):
        n = self.n_cells
        outs = [np.zeros(n) for _ in range(3)]
        u, v, w = _f64(u), _f64(v), _f64(w)
        ubk = _f64(ub) if ub is not None and np.size(ub) else None
        lib().orc_convection_quick(self._h, _p(u), _p(v), _p(w),
                                   _p(ubk) if ubk is not None else None, *[_p(o) for o in outs])
        return outs

    def set_scheme(self, scheme: int, cn_rtol: float = 1e-10, cn_max: int = 100):
        """Momentum scheme of the following steps: 0 AB2 + central, 1 QUICK + CN."""
        if lib().orc_set_scheme(self._h, scheme, cn_rtol, cn_max):
            raise ValueError(lib().orc_error().decode())

    # ------------------------------------------------ Lagrangian particles (R19)
    @staticmethod
    def delta3(r: float) -> float:
        return lib().orc_delta3(float(r))

    def ib_interpolate(self, f, parts) -> np.ndarray:
        """I[f] at every particle of a workloads.Particles set (Eq. ddeltai)."""
        f = _f64(f)
        X, sim = _f64(parts.X), np.ascontiguousarray(parts.sim, np.int32)
        out = np.zeros(parts.n)
        lib().orc_ib_interpolate(self._h, _p(f), parts.n, _p(X), _p(sim), _p(out))
        return out

    def ib_spread(self, F, parts, out=None) -> np.ndarray:
        """out += P[F] (Eq. ddeltap), F one value per particle."""
        out = np.zeros(self.n_cells) if out is None else out
        F = _f64(F)
        X, sim, dV = _f64(parts.X), np.ascontiguousarray(parts.sim, np.int32), _f64(parts.dV)
        lib().orc_ib_spread(self._h, parts.n, _p(X), _p(sim), _p(F), _p(dV), _p(out))
        return out

    def ib_body_velocity(self, X, parts, t) -> np.ndarray:
        X = _f64(X)
        sim = np.ascontiguousarray(parts.sim, np.int32)
        body = np.ascontiguousarray(parts.body, np.int32)
        t = _f64(np.broadcast_to(np.asarray(t, np.float64), (self.spec.n_sims,)))
        vel = np.zeros((parts.n, 3))
        lib().orc_ib_body_velocity(self._h, parts.n, _p(X), _p(sim), _p(body), _p(t), _p(vel))
        return vel

    def step_particles(self, st, X, parts, nsteps=1, rtol=1e-12, max_iter=100000):
        """Steps with the particle forcing; X ([n, 3] float64) is advanced in place.
        Returns (stats, rc, F) with F the last step's force per particle [n, 3]."""
        stats = (Stats * self.spec.n_sims)()
        ub = st["ub"]
        if ub.size == 0:
            ub = np.zeros(1)
            st["ub"] = ub
        assert X.dtype == np.float64 and X.flags.c_contiguous and X.shape == (parts.n, 3)
        sim = np.ascontiguousarray(parts.sim, np.int32)
        body = np.ascontiguousarray(parts.body, np.int32)
        dV = _f64(parts.dV)
        F = np.zeros((parts.n, 3))
        rc = lib().orc_step_particles(self._h, _p(st["u"]), _p(st["v"]), _p(st["w"]),
                                      _p(st["p"]), _p(st["nx"]), _p(st["ny"]), _p(st["nz"]),
                                      _p(ub), _p(st["step"]), nsteps, rtol, max_iter, stats,
                                      parts.n, _p(X), _p(sim), _p(body), _p(dV), _p(F))
        return [s.as_dict() for s in stats], rc, F

    @staticmethod
    def threads() -> int:
        return lib().orc_threads()

    @staticmethod
    def set_threads(n: int) -> int:
        """Threads of the oracle's parallel loops from now on; returns the previous count."""
        return lib().orc_set_threads(int(n))
