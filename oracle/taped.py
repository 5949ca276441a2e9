"""Taped restatement of the fractional step, for gradients.  Test infrastructure only:
tests import it; the library never does.

It uses plain PyTorch CPU float64 operations on one uniform single-level channel, with
one (z, y, x) array per field, so torch.autograd records the whole run and
differentiates it exactly.  It restates what the C oracle computes (the readings
R1-R8 and R14 in bcm_oracle.c) for the grids the adjoint step supports:
  * one sim on one level;
  * inflow with its profile modes at -x, convective outflow at +x, slip on y and z;
  * one fixed sphere.
It shares no code with the C oracle or the CUDA path: the cube structure is gone,
neighbours are array shifts, and the Poisson equation K p = -V b (Eq. poisson) is
solved with a dense LU factorisation of K (the library step is torch.linalg.lu_solve),
so grids stay at a few thousand cells.

Step n (section "Numerical algorithm": Eq. substep1, Eq. poisson, the projection)
from u^n, N^{n-1} and the outflow face values u_b^n:
  (a) the solid fraction phi = (1 - tanh(d / 1.5h)) / 2 of the sphere's signed distance
      d, and 0 from d = 20 (1.5h) on; the body velocity is 0;
  (b) one ghost layer of u^n:
      - x-: 2 U_in(y, z) - u;
      - x+: 2 u_b - u;
      - slip faces: the mirror value, negated for the normal component;
  (c) u~ = u^n + dt (-(3/2 N^n - 1/2 N^{n-1}) + nu L u^n), with N^{-1} = N^0.
      N is the flux form of central convection (face velocity times face value, both
      cell means) and L the 7-point Laplacian.  Then u* = u~ + phi (0 - u~), and the
      drag F = -sum (u* - u~) h^3 / dt;
  (d) u_b^{n+1} = u_b^n - U_c dt (u_b^n - u_adjacent^n) / (h/2);
  (e) b = div(u*) / dt.  Face velocities are cell means inside, U_in at x-,
      u_b^{n+1} at x+ and 0 through slip faces;
  (f) K p = -h^3 b.  K takes (h) (p_i - p_nb) per interior face and 2h p_i at the
      outflow face (p = 0 there); Neumann faces add nothing;
  (g) u^{n+1} = u* - dt times the mean of the cell's two face gradients of p along each
      axis; a Neumann face's gradient is 0, the outflow face's -2 p / h.
J = (1/N) sum_n F_x^n, the time-averaged drag (R14).
"""
from __future__ import annotations

import numpy as np
import torch

from paper_1808_04099_gb300 import workloads as W

# (k, l) wave numbers of the eight inflow-profile modes in y and z
MODE_K = (1, 1, 2, 2, 1, 3, 2, 3)
MODE_L = (1, 2, 1, 2, 3, 1, 3, 2)

_F64 = torch.float64


def _inner(P, axis: int, shift: int):
    """Interior view of a one-layer padded (z, y, x) array, shifted by `shift` cells
    along `axis` (0 = x, 1 = y, 2 = z)."""
    sl = [slice(1, -1)] * 3
    dim = 2 - axis
    n = P.shape[dim]
    sl[dim] = slice(1 + shift, n - 1 + shift)
    return P[tuple(sl)]


class TapedChannel:
    """The channel of `spec` (W.sphere_channel layout), steps restated in torch."""

    def __init__(self, spec: W.GridSpec):
        if spec.n_sims != 1 or spec.max_level != 0:
            raise ValueError("one sim on one level")
        if list(spec.sim_bc[0]) != [W.INFLOW, W.OUTFLOW, W.SLIP, W.SLIP, W.SLIP, W.SLIP]:
            raise ValueError("inflow -x, outflow +x, slip on y and z")
        self.spec = spec
        self.B = spec.B
        self.nx, self.ny, self.nz = (int(e) for e in spec.sim_extent[0])
        self.h = float(spec.sim_h0[0])
        self.dt = float(spec.sim_dt[0])
        self.nu = float(spec.sim_nu[0])
        self.uc = float(spec.sim_uconv[0])
        self.u_in = np.asarray(spec.sim_bc_vel[0, 0], np.float64)
        o = np.asarray(spec.sim_origin[0], np.float64)
        h = self.h
        self.xc = torch.tensor(o[0] + (np.arange(self.nx) + 0.5) * h, dtype=_F64)
        self.yc = torch.tensor(o[1] + (np.arange(self.ny) + 0.5) * h, dtype=_F64)
        self.zc = torch.tensor(o[2] + (np.arange(self.nz) + 0.5) * h, dtype=_F64)
        self.Ly, self.Lz = self.ny * h, self.nz * h
        self.lu = torch.linalg.lu_factor(torch.tensor(self._poisson_matrix(), dtype=_F64))

    # ------------------------------------------------------------ layout maps
    def to_grid(self, f) -> np.ndarray:
        """Cube-major cell field -> (z, y, x) array."""
        B = self.B
        out = np.empty((self.nz, self.ny, self.nx))
        cubes = np.asarray(f, np.float64).reshape(-1, B, B, B)
        for c, (ci, cj, ck) in enumerate(self.spec.cube_ijk):
            out[ck:ck + B, cj:cj + B, ci:ci + B] = cubes[c]
        return out

    def ub_to_grid(self, ub) -> np.ndarray:
        """Outflow face values [slot, comp, b, a] -> [comp, z, y] on the +x face."""
        B = self.B
        out = np.empty((3, self.nz, self.ny))
        for sl, (c, f) in enumerate(W.outflow_slots(self.spec)):
            _, cj, ck = self.spec.cube_ijk[c]
            out[:, ck:ck + B, cj:cj + B] = np.asarray(ub).reshape(-1, 3, B, B)[sl]
        return out

    # ------------------------------------------------------------- operators
    def _poisson_matrix(self) -> np.ndarray:
        nx, ny, nz, h = self.nx, self.ny, self.nz, self.h
        n = nx * ny * nz
        K = np.zeros((n, n))
        idx = np.arange(n).reshape(nz, ny, nx)
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    r = idx[k, j, i]
                    for (di, dj, dk) in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                                         (0, 0, 1), (0, 0, -1)):
                        a, b, c = i + di, j + dj, k + dk
                        if 0 <= a < nx and 0 <= b < ny and 0 <= c < nz:
                            K[r, r] += h
                            K[r, idx[c, b, a]] -= h
                        elif a == nx:  # outflow face: p = 0 on it
                            K[r, r] += 2.0 * h
        return K

    def inflow_profile(self, modes):
        """1 + sum_m a_m sin(k_m pi y / L_y) sin(l_m pi z / L_z) on the x- face, (z, y)."""
        y = self.yc[None, :] - float(self.spec.sim_origin[0][1])
        z = self.zc[:, None] - float(self.spec.sim_origin[0][2])
        prof = torch.ones((self.nz, self.ny), dtype=_F64)
        for m in range(8):
            prof = prof + modes[m] * torch.sin(MODE_K[m] * np.pi * y / self.Ly) * \
                torch.sin(MODE_L[m] * np.pi * z / self.Lz)
        return prof

    def solid_fraction(self, center, radius: float):
        eps = 1.5 * self.h
        d = torch.sqrt((self.xc[None, None, :] - center[0]) ** 2 +
                       (self.yc[None, :, None] - center[1]) ** 2 +
                       (self.zc[:, None, None] - center[2]) ** 2) - radius
        return torch.where(d < 20.0 * eps, 0.5 * (1.0 - torch.tanh(d / eps)),
                           torch.zeros_like(d))

    def _pad(self, f, comp: int, u_face_in, ub_c):
        """One ghost layer of velocity component `comp` (rule (b))."""
        nz, ny, nx = f.shape
        P = torch.zeros((nz + 2, ny + 2, nx + 2), dtype=_F64)
        P[1:-1, 1:-1, 1:-1] = f
        P[1:-1, 1:-1, 0] = 2.0 * u_face_in - f[:, :, 0]
        P[1:-1, 1:-1, -1] = 2.0 * ub_c - f[:, :, -1]
        sy = -1.0 if comp == 1 else 1.0
        P[1:-1, 0, 1:-1] = sy * f[:, 0, :]
        P[1:-1, -1, 1:-1] = sy * f[:, -1, :]
        sz = -1.0 if comp == 2 else 1.0
        P[0, 1:-1, 1:-1] = sz * f[0, :, :]
        P[-1, 1:-1, 1:-1] = sz * f[-1, :, :]
        return P

    def _conv_diff(self, Ps, comp: int):
        """N (central flux form) and L of component comp from the padded fields."""
        h = self.h
        uc = Ps[comp]
        u0 = _inner(uc, 0, 0)
        N = torch.zeros_like(u0)
        L = torch.zeros_like(u0)
        for d in range(3):
            ud = Ps[d]
            up, um = _inner(uc, d, 1), _inner(uc, d, -1)
            vd0, vdp, vdm = _inner(ud, d, 0), _inner(ud, d, 1), _inner(ud, d, -1)
            N = N + (0.5 * (vd0 + vdp) * 0.5 * (u0 + up) - 0.5 * (vdm + vd0) * 0.5 * (um + u0))
            L = L + (up - 2.0 * u0 + um)
        return N / h, L / (h * h)

    def _divergence(self, us, ubn, u_face_in):
        """sum over faces of the outward normal face velocity (rule (e)), per cell."""
        ux, uy, uz = us
        zero_y = torch.zeros_like(uy[:, :1, :])
        zero_z = torch.zeros_like(uz[:1, :, :])
        fx = torch.cat([u_face_in[:, :, None], 0.5 * (ux[:, :, 1:] + ux[:, :, :-1]),
                        ubn[0][:, :, None]], dim=2)
        fy = torch.cat([zero_y, 0.5 * (uy[:, 1:, :] + uy[:, :-1, :]), zero_y], dim=1)
        fz = torch.cat([zero_z, 0.5 * (uz[1:, :, :] + uz[:-1, :, :]), zero_z], dim=0)
        return (fx[:, :, 1:] - fx[:, :, :-1]) + (fy[:, 1:, :] - fy[:, :-1, :]) + \
            (fz[1:, :, :] - fz[:-1, :, :])

    def _gradient(self, p):
        """Mean of the two face gradients along each axis (rule (g))."""
        h = self.h
        zy = torch.zeros_like(p[:, :1, :])
        zz = torch.zeros_like(p[:1, :, :])
        gx = torch.cat([torch.zeros_like(p[:, :, :1]), (p[:, :, 1:] - p[:, :, :-1]) / h,
                        -2.0 * p[:, :, -1:] / h], dim=2)
        gy = torch.cat([zy, (p[:, 1:, :] - p[:, :-1, :]) / h, zy], dim=1)
        gz = torch.cat([zz, (p[1:, :, :] - p[:-1, :, :]) / h, zz], dim=0)
        return (0.5 * (gx[:, :, 1:] + gx[:, :, :-1]), 0.5 * (gy[:, 1:, :] + gy[:, :-1, :]),
                0.5 * (gz[1:, :, :] + gz[:-1, :, :]))

    # ------------------------------------------------------------------ run
    def run(self, modes, center, radius: float, steps: int, state: W.State):
        """Steps from `state`; returns (J, per-step drag [steps, 3], final (u, v, w, p),
        final outflow face values).  modes and center may be tensors that require grad."""
        modes = torch.as_tensor(modes, dtype=_F64)
        center = torch.as_tensor(center, dtype=_F64)
        dt, nu, h = self.dt, self.nu, self.h
        V = h ** 3
        u = [torch.tensor(self.to_grid(f), dtype=_F64) for f in (state.u, state.v, state.w)]
        ub = torch.tensor(self.ub_to_grid(state.ub), dtype=_F64)
        prof = self.inflow_profile(modes)
        u_face = [float(self.u_in[c]) * prof for c in range(3)]
        phi = self.solid_fraction(center, radius)  # fixed sphere: the same every step
        n_prev = None
        drags = []
        p = None
        for _ in range(steps):
            Ps = [self._pad(u[c], c, u_face[c], ub[c]) for c in range(3)]
            ubn = ub - self.uc * dt * (ub - torch.stack([u[c][:, :, -1] for c in range(3)])) \
                / (0.5 * h)
            N, L, us, F = [], [], [], []
            for c in range(3):
                Nc, Lc = self._conv_diff(Ps, c)
                Np = Nc if n_prev is None else n_prev[c]
                ut = u[c] + dt * (-(1.5 * Nc - 0.5 * Np) + nu * Lc)
                du = phi * (0.0 - ut)
                us.append(ut + du)
                F.append(-(du / dt).sum() * V)
                N.append(Nc)
            drags.append(torch.stack(F))
            b = self._divergence(us, ubn, u_face[0]) / (h * dt)
            rhs = (-V * b).reshape(-1, 1)
            p = torch.linalg.lu_solve(self.lu[0], self.lu[1], rhs).reshape(b.shape)
            gx, gy, gz = self._gradient(p)
            u = [us[0] - dt * gx, us[1] - dt * gy, us[2] - dt * gz]
            ub = ubn
            n_prev = N
        drag = torch.stack(drags)
        J = drag[:, 0].sum() / steps
        return J, drag, (u[0], u[1], u[2], p), ub


def drag_gradient(spec: W.GridSpec, modes, center, radius: float, steps: int, state=None):
    """J and dJ/d(modes, centre) of the time-averaged drag by reverse-mode autograd."""
    tc = TapedChannel(spec)
    a = torch.tensor(np.asarray(modes, np.float64), requires_grad=True)
    c = torch.tensor(np.asarray(center, np.float64), requires_grad=True)
    st = state if state is not None else W.initial_state(spec)
    J, _, _, _ = tc.run(a, c, radius, steps, st)
    J.backward()
    return float(J.detach()), a.grad.numpy().copy(), c.grad.numpy().copy()
