"""Python binding of libbcm.so (include/bcm.h): argument marshalling only.

PyTorch provides the device workspace (one uint8 tensor) and the CUDA stream;
every step of the time step runs in the library's kernels.  There is no CPU or
PyTorch fallback: if the library cannot be built or loaded, this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional

import numpy as np

from . import _build

# status codes
BCM_OK, BCM_E_INVALID, BCM_E_CUDA, BCM_E_NOT_CONVERGED = 0, -1, -2, -3
BCM_E_NONFINITE, BCM_E_TIMEOUT, BCM_E_BOUNDS = -4, -5, -6
PREC_F64, PREC_F32_REFINE, PREC_F64_REFINE = 0, 1, 2
PRECOND_JACOBI, PRECOND_MULTIGRID = 0, 1
SCHEME_AB2_CENTRAL, SCHEME_QUICK_CN = 0, 1
(U, V, W, P, PHI, NX, NY, NZ, USTAR, VSTAR, WSTAR, RHS, UB) = range(13)

EXPORTED = ["bcm_workspace_bytes", "bcm_create_grid", "bcm_destroy_grid", "bcm_field",
            "bcm_set_geometry", "bcm_reset_time", "bcm_drag_mean", "bcm_set_solver",
            "bcm_set_launch", "bcm_set_stencil_slabs", "bcm_get_stencil_slabs",
            "bcm_set_preconditioner", "bcm_apply_preconditioner",
            "bcm_set_step", "bcm_get_solver", "bcm_measure_fma_rate", "bcm_step", "bcm_step_graph", "bcm_solve_pressure",
            "bcm_adjoint_bytes", "bcm_adjoint_init", "bcm_adjoint_step",
            "bcm_fill_halo", "bcm_apply_poisson", "bcm_solve_pressure_static",
            "bcm_profile", "bcm_profile_read",
            "bcm_set_momentum_scheme",
            "bcm_compress_bound", "bcm_compress_field", "bcm_decompress_field",
            "bcm_particles_bytes", "bcm_set_particles", "bcm_get_particles",
            "bcm_particle_sets", "bcm_ib_interpolate", "bcm_ib_spread",
            "bcm_last_error"]
KERNEL_NAMES = ["solid_fraction", "momentum", "rhs", "residual", "cg_a", "cg_b",
                "add_correction", "correct", "misc", "pcg", "mg", "ib"]


class GridDesc(C.Structure):
    _fields_ = [("n_sims", C.c_int32), ("n_cubes", C.c_int32), ("cells_per_edge", C.c_int32),
                ("max_level", C.c_int32), ("precision", C.c_int32), ("lagged_bf16", C.c_int32),
                ("sim_cube_offset", C.c_void_p), ("cube_ijk", C.c_void_p),
                ("cube_level", C.c_void_p), ("sim_extent", C.c_void_p),
                ("sim_origin", C.c_void_p), ("sim_h0", C.c_void_p), ("sim_bc", C.c_void_p),
                ("sim_bc_vel", C.c_void_p), ("sim_nu", C.c_void_p), ("sim_dt", C.c_void_p),
                ("sim_uconv", C.c_void_p)]


class Body(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("center", C.c_double * 3),
                ("axes", C.c_double * 3), ("quat", C.c_double * 4), ("omega", C.c_double * 3),
                ("vel", C.c_double * 3)]


class Stats(C.Structure):
    _fields_ = [("cg_iters", C.c_int32), ("refine_cycles", C.c_int32), ("steps", C.c_int32),
                ("converged", C.c_int32), ("rel_resid", C.c_double), ("div_rel", C.c_double),
                ("drag", C.c_double * 3), ("umax", C.c_double), ("pcg_form", C.c_int32),
                ("cn_iters", C.c_int32)]

    def as_dict(self):
        return {"cg_iters": self.cg_iters, "refine_cycles": self.refine_cycles,
                "steps": self.steps, "converged": self.converged, "rel_resid": self.rel_resid,
                "div_rel": self.div_rel, "drag": list(self.drag), "umax": self.umax,
                "pcg_form": self.pcg_form, "cn_iters": self.cn_iters}


class BCMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"bcm status {status}: {msg}")
        self.status = status


_lib = None


def lib(build: bool = True):
    """Load libbcm.so (building it in-tree first when sources are newer); with the
    environment variable BCM_CHECK=1, the checked build libbcm_check.so."""
    global _lib
    if _lib is None:
        check = os.environ.get("BCM_CHECK") == "1"
        if check:
            path = _build.build(check=True) if build else _build.LIB_CHECK
        else:
            path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libbcm.so is missing; run __graft_entry__.build()")
        L = C.CDLL(path)
        P = C.c_void_p
        L.bcm_workspace_bytes.restype = C.c_size_t
        L.bcm_workspace_bytes.argtypes = [P]
        L.bcm_create_grid.argtypes = [P, P, C.c_size_t, P, C.POINTER(C.c_void_p)]
        L.bcm_destroy_grid.argtypes = [P]
        L.bcm_field.argtypes = [P, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_size_t),
                                C.POINTER(C.c_int32)]
        L.bcm_set_geometry.argtypes = [P, C.c_int, P, C.c_int, P]
        L.bcm_reset_time.argtypes = [P]
        L.bcm_drag_mean.argtypes = [P, C.c_int, P]
        L.bcm_set_step.argtypes = [P, C.c_int]
        L.bcm_adjoint_bytes.restype = C.c_size_t
        L.bcm_adjoint_bytes.argtypes = [P]
        L.bcm_adjoint_init.argtypes = [P, P, C.c_size_t]
        L.bcm_adjoint_step.argtypes = [P, P, C.c_size_t, P, C.c_int, C.c_double, C.c_double,
                                       C.c_int, P]
        L.bcm_set_solver.argtypes = [P, C.c_double, C.c_int, C.c_int, C.c_double, C.c_int]
        L.bcm_set_launch.argtypes = [P, C.c_int, C.c_int, C.c_int]
        L.bcm_set_stencil_slabs.argtypes = [P, C.c_int]
        L.bcm_get_stencil_slabs.argtypes = [P, P]
        L.bcm_get_solver.argtypes = [P, P, P, P, P, P]
        L.bcm_measure_fma_rate.argtypes = [C.c_int, P]
        L.bcm_step.argtypes = [P, C.c_int, C.c_double, C.c_int, P]
        L.bcm_step_graph.argtypes = [P, C.c_int, C.c_double, C.c_int, P]
        L.bcm_solve_pressure.argtypes = [P, C.c_double, C.c_int, P]
        L.bcm_fill_halo.argtypes = [P, C.c_int, C.c_int, P]
        L.bcm_apply_poisson.argtypes = [P, P, P]
        L.bcm_set_preconditioner.argtypes = [P, C.c_int]
        L.bcm_apply_preconditioner.argtypes = [P, P, P]
        L.bcm_solve_pressure_static.argtypes = [P, P, P, C.c_double, C.c_int, P]
        L.bcm_profile.argtypes = [P, C.c_int]
        L.bcm_profile_read.argtypes = [P, P, P, P, C.c_int]
        L.bcm_set_momentum_scheme.argtypes = [P, C.c_int, C.c_double, C.c_int]
        L.bcm_compress_bound.restype = C.c_size_t
        L.bcm_compress_bound.argtypes = [P]
        L.bcm_compress_field.argtypes = [P, C.c_int, C.c_double, P, C.c_size_t,
                                         C.POINTER(C.c_size_t)]
        L.bcm_decompress_field.argtypes = [P, C.c_int, P, C.c_size_t]
        L.bcm_particles_bytes.restype = C.c_size_t
        L.bcm_particles_bytes.argtypes = [P, C.c_int32]
        L.bcm_set_particles.argtypes = [P, C.c_int32, P, P, P, P, P, C.c_size_t]
        L.bcm_get_particles.argtypes = [P, P, P, P]
        L.bcm_particle_sets.argtypes = [P, P, P]
        L.bcm_ib_interpolate.argtypes = [P, P, P]
        L.bcm_ib_spread.argtypes = [P, P, P]
        L.bcm_last_error.restype = C.c_char_p
        for name in EXPORTED:
            if name not in ("bcm_adjoint_bytes", "bcm_particles_bytes", "bcm_compress_bound"):
                getattr(L, name).restype = getattr(L, name).restype or C.c_int
        _lib = L
    return _lib


def _check(rc: int, allow=()):
    if rc != BCM_OK and rc not in allow:
        raise BCMError(rc, lib().bcm_last_error().decode())
    return rc


def _body_struct(b) -> Body:
    s = Body()
    s.kind = int(b.kind)
    s.center[:] = list(map(float, b.center))
    s.axes[:] = list(map(float, b.axes))
    s.quat[:] = list(map(float, b.quat))
    s.omega[:] = list(map(float, b.omega))
    s.vel[:] = list(map(float, b.vel))
    return s


def fma_rate(fp64: bool = True) -> float:
    """Measured FMA rate of the current device in FLOP/s (FP64 or FP32)."""
    r = C.c_double()
    _check(lib().bcm_measure_fma_rate(1 if fp64 else 0, C.byref(r)))
    return r.value


class Grid:
    """One BCM grid (one or more independent sims) living in a torch-owned workspace."""

    def __init__(self, spec, precision: int = PREC_F64, device=None, stream=None,
                 lagged_bf16: bool = False):
        """lagged_bf16: in mixed precision, store the lagged convection N^{n-1} (fields
        NX, NY, NZ) as bfloat16."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the BCM library needs a CUDA device")
        L = lib()
        self.spec = spec
        self.precision = precision
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self._arrays = [np.ascontiguousarray(spec.sim_cube_offset, np.int32),
                        np.ascontiguousarray(spec.cube_ijk, np.int32),
                        np.ascontiguousarray(spec.cube_level, np.int8),
                        np.ascontiguousarray(spec.sim_extent, np.int32),
                        np.ascontiguousarray(spec.sim_origin, np.float64),
                        np.ascontiguousarray(spec.sim_h0, np.float64),
                        np.ascontiguousarray(spec.sim_bc, np.int32),
                        np.ascontiguousarray(spec.sim_bc_vel, np.float64),
                        np.ascontiguousarray(spec.sim_nu, np.float64),
                        np.ascontiguousarray(spec.sim_dt, np.float64),
                        np.ascontiguousarray(spec.sim_uconv, np.float64)]
        d = GridDesc()
        d.n_sims, d.n_cubes, d.cells_per_edge = spec.n_sims, spec.n_cubes, spec.B
        d.max_level, d.precision = spec.max_level, precision
        d.lagged_bf16 = 1 if lagged_bf16 else 0
        (d.sim_cube_offset, d.cube_ijk, d.cube_level, d.sim_extent, d.sim_origin, d.sim_h0,
         d.sim_bc, d.sim_bc_vel, d.sim_nu, d.sim_dt, d.sim_uconv) = \
            [a.ctypes.data for a in self._arrays]
        self._desc = d
        nbytes = L.bcm_workspace_bytes(C.byref(d))
        if nbytes == 0:
            raise BCMError(BCM_E_INVALID, L.bcm_last_error().decode())
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            base = self.workspace.data_ptr()
            self._off0 = (-base) % 256
            self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
            h = C.c_void_p()
            _check(L.bcm_create_grid(C.byref(d), C.c_void_p(base + self._off0), nbytes,
                                     C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h
        self.nbytes = nbytes
        for s, bodies in enumerate(spec.bodies):
            if bodies or np.any(spec.inflow_modes[s]):
                self.set_geometry(s, bodies, spec.inflow_modes[s])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.bcm_destroy_grid(h)
            self._h = None

    # ------------------------------------------------------------------ fields
    def field(self, fid: int):
        """Zero-copy torch view of one field (shares the workspace)."""
        import torch
        ptr, cnt, eb = C.c_void_p(), C.c_size_t(), C.c_int32()
        _check(lib().bcm_field(self._h, fid, C.byref(ptr), C.byref(cnt), C.byref(eb)))
        off = ptr.value - self.workspace.data_ptr()
        n = cnt.value * eb.value
        dt = {8: torch.float64, 4: torch.float32, 2: torch.bfloat16}[eb.value]
        return self.workspace[off:off + n].view(dt)

    def load_state(self, state):
        """Copy a workloads.State (host arrays) into the grid's fields."""
        import torch
        for fid, arr in ((U, state.u), (V, state.v), (W, state.w), (P, state.p)):
            t = self.field(fid)
            t.copy_(torch.as_tensor(np.asarray(arr).reshape(-1)).to(t.dtype))
        ub = self.field(UB)
        if ub.numel():
            ub.copy_(torch.as_tensor(np.asarray(state.ub).reshape(-1)).to(ub.dtype))
        for fid in (NX, NY, NZ):
            self.field(fid).zero_()
        self.reset_time()

    def numpy(self, fid: int) -> np.ndarray:
        import torch
        torch.cuda.current_stream(self.device).synchronize()
        self.stream.synchronize()
        return self.field(fid).double().cpu().numpy()

    # -------------------------------------------------------------- operations
    def set_geometry(self, sim: int, bodies, modes=None):
        arr = (Body * max(1, len(bodies)))(*[_body_struct(b) for b in bodies])
        m = None if modes is None else np.ascontiguousarray(modes, np.float64)
        _check(lib().bcm_set_geometry(self._h, sim, arr if bodies else None, len(bodies),
                                      m.ctypes.data if m is not None else None))

    def set_solver(self, inner_rtol: float = 0.0, max_cycles: int = 0, check_every: int = 0,
                   barrier_timeout_s: float = 0.0, recycle: int = -1):
        _check(lib().bcm_set_solver(self._h, inner_rtol, max_cycles, check_every,
                                    barrier_timeout_s, recycle))

    def get_solver(self) -> dict:
        """The solver controls in effect (inner_rtol 0 = automatic)."""
        ir, bt = C.c_double(), C.c_double()
        mc, ce, rc = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().bcm_get_solver(self._h, C.byref(ir), C.byref(mc), C.byref(ce),
                                    C.byref(bt), C.byref(rc)))
        return {"inner_rtol": ir.value, "max_cycles": mc.value, "check_every": ce.value,
                "barrier_timeout_s": bt.value, "recycle": rc.value}

    def set_preconditioner(self, kind: int):
        """PRECOND_JACOBI (default) or PRECOND_MULTIGRID."""
        _check(lib().bcm_set_preconditioner(self._h, int(kind)))

    def apply_preconditioner(self, r):
        """z = M^-1 r by one multigrid V-cycle (FP64 grids; test path)."""
        import torch
        r = torch.as_tensor(r).to(self.device, torch.float64).contiguous()
        z = torch.empty_like(r)
        _check(lib().bcm_apply_preconditioner(self._h, C.c_void_p(r.data_ptr()),
                                              C.c_void_p(z.data_ptr())))
        return z

    def set_momentum_scheme(self, scheme: int, cn_rtol: float = 0.0, cn_max_iter: int = 0):
        """SCHEME_AB2_CENTRAL (default) or SCHEME_QUICK_CN (0: library defaults)."""
        _check(lib().bcm_set_momentum_scheme(self._h, int(scheme), float(cn_rtol),
                                             int(cn_max_iter)))

    # ------------------------------------------------ wavelet compression
    def compress_field(self, fid: int, step: float):
        """Wavelet stream of one cell field (a uint32 device tensor of the stream words)."""
        import torch
        cap = lib().bcm_compress_bound(self._h)
        buf = torch.empty(cap // 4, dtype=torch.int32, device=self.device)
        n = C.c_size_t()
        _check(lib().bcm_compress_field(self._h, int(fid), float(step),
                                        C.c_void_p(buf.data_ptr()), cap, C.byref(n)))
        return buf[:n.value // 4].clone()

    def decompress_field(self, fid: int, stream):
        """Decode a stream of compress_field into the field."""
        import torch
        stream = torch.as_tensor(stream).to(self.device).contiguous()
        _check(lib().bcm_decompress_field(self._h, int(fid), C.c_void_p(stream.data_ptr()),
                                          stream.numel() * stream.element_size()))

    # ------------------------------------------------ Lagrangian particles
    def set_particles(self, parts):
        """Lagrangian-particle IB with a workloads.Particles set (None or an empty set:
        back to the solid fraction).  The particle workspace is a torch tensor kept
        alive by the grid."""
        import torch
        L = lib()
        n = 0 if parts is None else int(parts.n)
        if n == 0:
            _check(L.bcm_set_particles(self._h, 0, None, None, None, None, None, 0))
            self._pws = None
            return
        nbytes = L.bcm_particles_bytes(self._h, n)
        if nbytes == 0:
            raise BCMError(BCM_E_INVALID, "particles need a single-level grid")
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-ws.data_ptr()) % 256
        X = np.ascontiguousarray(parts.X, np.float64)
        sim = np.ascontiguousarray(parts.sim, np.int32)
        body = np.ascontiguousarray(parts.body, np.int32)
        dV = np.ascontiguousarray(parts.dV, np.float64)
        self.stream.synchronize()
        _check(L.bcm_set_particles(self._h, n, X.ctypes.data, sim.ctypes.data, body.ctypes.data,
                                   dV.ctypes.data, C.c_void_p(ws.data_ptr() + off), nbytes))
        self._pws = ws
        self._np = n

    def particles(self):
        """(positions [n, 3], last step's force per particle [n, 3], cube per particle)."""
        n = getattr(self, "_np", 0) if getattr(self, "_pws", None) is not None else 0
        X, F = np.zeros((n, 3)), np.zeros((n, 3))
        cube = np.zeros(n, np.int32)
        _check(lib().bcm_get_particles(self._h, X.ctypes.data, F.ctypes.data, cube.ctypes.data))
        return X, F, cube

    def particle_sets(self):
        """Per-cube sets: (start [n_cubes + 1], ids [n])."""
        start = np.zeros(self.spec.n_cubes + 1, np.int32)
        ids = np.zeros(self._np, np.int32)
        _check(lib().bcm_particle_sets(self._h, start.ctypes.data, ids.ctypes.data))
        return start, ids

    def ib_interpolate(self, f):
        """I[f] at every particle (FP64 test path)."""
        import torch
        f = torch.as_tensor(f).to(self.device, torch.float64).contiguous()
        out = torch.zeros(self._np, dtype=torch.float64, device=self.device)
        _check(lib().bcm_ib_interpolate(self._h, C.c_void_p(f.data_ptr()),
                                        C.c_void_p(out.data_ptr())))
        return out

    def ib_spread(self, F):
        """P[F] on the cells, F one value per particle (FP64 test path)."""
        import torch
        F = torch.as_tensor(F).to(self.device, torch.float64).contiguous()
        out = torch.zeros(self.spec.n_cells, dtype=torch.float64, device=self.device)
        _check(lib().bcm_ib_spread(self._h, C.c_void_p(F.data_ptr()),
                                   C.c_void_p(out.data_ptr())))
        return out

    def set_launch(self, slabs_a: int = 1, slabs_b: int = 1, persistent: int = 1):
        """persistent: 0 two launches per iteration, 1 the persistent two-pass PCG
        streaming its vectors through global memory, 2 the persistent single-reduction
        PCG, 3 the persistent two-pass PCG with the search direction in shared memory
        where the grid fits one co-resident wave, 5 the fused single-barrier PCG (mixed
        precision on 16^3 cubes, else the two-pass form runs; bool values map to 0 and
        1)."""
        _check(lib().bcm_set_launch(self._h, int(persistent), slabs_a, slabs_b))

    def set_stencil_slabs(self, slabs: int):
        """z-slabs per 16^3 cube of the momentum and right-hand-side kernels (1, 2, 4; 0:
        the default)."""
        _check(lib().bcm_set_stencil_slabs(self._h, int(slabs)))

    def get_stencil_slabs(self) -> int:
        v = C.c_int32()
        _check(lib().bcm_get_stencil_slabs(self._h, C.byref(v)))
        return v.value

    def set_step(self, step: int):
        _check(lib().bcm_set_step(self._h, step))

    def reset_time(self):
        _check(lib().bcm_reset_time(self._h))

    def drag_mean(self, reset: bool = False) -> np.ndarray:
        """[n_sims, 3]: the mean per-step drag since the last reset (reset: start anew)."""
        out = np.zeros((self.spec.n_sims, 3), np.float64)
        _check(lib().bcm_drag_mean(self._h, int(reset), out.ctypes.data_as(C.c_void_p)))
        return out

    def step(self, n: int = 1, rtol: float = 1e-10, max_iter: int = 20000, stats: bool = True,
             allow_not_converged: bool = False) -> Optional[List[dict]]:
        st = (Stats * self.spec.n_sims)() if stats else None
        rc = lib().bcm_step(self._h, n, rtol, max_iter, st)
        _check(rc, (BCM_E_NOT_CONVERGED,) if allow_not_converged else ())
        return [s.as_dict() for s in st] if stats else None

    def step_graph(self, n: int = 1, rtol: float = 1e-10, max_iter: int = 20000,
                   stats: bool = True, allow_not_converged: bool = False):
        """n steps by replaying a captured CUDA graph of one step."""
        st = (Stats * self.spec.n_sims)() if stats else None
        rc = lib().bcm_step_graph(self._h, n, rtol, max_iter, st)
        _check(rc, (BCM_E_NOT_CONVERGED,) if allow_not_converged else ())
        return [s.as_dict() for s in st] if stats else None

    def solve_pressure(self, rtol: float = 1e-12, max_iter: int = 20000):
        st = (Stats * self.spec.n_sims)()
        _check(lib().bcm_solve_pressure(self._h, rtol, max_iter, st))
        return [s.as_dict() for s in st]

    def profile(self, enable: bool):
        _check(lib().bcm_profile(self._h, int(enable)))

    def profile_read(self, reset: bool = True):
        """{kernel: (total_ms, timed_launches)} and the count of all launches."""
        ms = (C.c_double * len(KERNEL_NAMES))()
        n = (C.c_int64 * len(KERNEL_NAMES))()
        total = C.c_int64()
        _check(lib().bcm_profile_read(self._h, ms, n, C.byref(total), int(reset)))
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_NAMES)}, total.value

    def solve_pressure_iters(self, iters: int):
        """Run exactly `iters` PCG iterations on the current right-hand side (timing aid:
        the tolerance is set out of reach, the not-converged status is expected)."""
        st = (Stats * self.spec.n_sims)()
        _check(lib().bcm_solve_pressure(self._h, 1e-300, iters, st), (BCM_E_NOT_CONVERGED,))
        return [s.as_dict() for s in st]

    def fill_halo(self, fid: int, kind: int):
        import torch
        G = self.spec.B + 4
        out = torch.zeros(self.spec.n_cubes * G ** 3, dtype=torch.float64, device=self.device)
        _check(lib().bcm_fill_halo(self._h, fid, kind, C.c_void_p(out.data_ptr())))
        return out

    def apply_poisson(self, x):
        import torch
        x = x.to(self.device, torch.float64).contiguous()
        y = torch.empty_like(x)
        _check(lib().bcm_apply_poisson(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr())))
        return y
