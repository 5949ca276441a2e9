"""Drag gradients by the discrete adjoint of the fractional step (bcm_adjoint_*).

J = (1/N) sum_{n<N} F_x^n, the time-averaged drag on a fixed sphere over N steps,
as a function of the eight inflow-profile amplitudes a and the sphere centre c.
The forward run keeps checkpoints of the state every `checkpoint_every` steps; the
backward sweep restores each segment's checkpoint, recomputes the segment's states
with the forward kernels and reverses its steps with the adjoint kernels.  This
module only orchestrates: every arithmetic step runs in libbcm's kernels, torch only
holds device memory (workspaces and state snapshots).
"""
from __future__ import annotations

import copy
import ctypes as C
from typing import List, Tuple

import numpy as np

from . import bcm
from . import workloads as W

STATE_FIELDS = (bcm.U, bcm.V, bcm.W, bcm.NX, bcm.NY, bcm.NZ, bcm.UB, bcm.P)


def _snapshot(g):
    return [g.field(f).clone() for f in STATE_FIELDS]


def _restore(g, snap):
    for f, t in zip(STATE_FIELDS, snap):
        g.field(f).copy_(t)


class AdjointRun:
    """A forward FP64 run with checkpoints, and its reverse sweep."""

    def __init__(self, spec, modes, center, radius: float, steps: int,
                 checkpoint_every: int = 10, rtol: float = 1e-12, max_iter: int = 50000,
                 state=None):
        import torch
        self.spec = copy.deepcopy(spec)
        self.modes = np.asarray(modes, np.float64).reshape(8)
        self.center = np.asarray(center, np.float64).reshape(3)
        self.spec.inflow_modes = self.modes[None, :].copy()
        self.spec.bodies = [[W.Body(W.BODY_SPHERE, self.center.copy(), np.array([radius] * 3))]]
        self.steps = steps
        self.K = max(1, checkpoint_every)
        self.rtol = rtol
        self.max_iter = max_iter
        self.g = bcm.Grid(self.spec, bcm.PREC_F64)
        self.g.set_launch(1, 1, persistent=False)
        self.state0 = state if state is not None else W.initial_state(self.spec)
        L = bcm.lib()
        self.adj_bytes = L.bcm_adjoint_bytes(self.g._h)
        self.adj = torch.zeros(self.adj_bytes + 256, dtype=torch.uint8, device=self.g.device)
        self._adj_off = (-self.adj.data_ptr()) % 256
        self.dJ = torch.zeros(11, dtype=torch.float64, device=self.g.device)
        self.J = None
        self.checkpoints = {}

    def forward(self) -> float:
        g = self.g
        g.load_state(self.state0)
        g.set_step(0)
        g.drag_mean(reset=True)  # J: the library's mean of the steps' drag
        for n in range(self.steps):
            if n % self.K == 0:
                self.checkpoints[n] = _snapshot(g)
            g.step(1, rtol=self.rtol, max_iter=self.max_iter)
        self.J = float(g.drag_mean()[0, 0])
        return self.J

    def backward(self) -> Tuple[np.ndarray, np.ndarray]:
        """dJ/da (8) and dJ/dc (3)."""
        L = bcm.lib()
        g = self.g
        adj_ptr = C.c_void_p(self.adj.data_ptr() + self._adj_off)
        bcm._check(L.bcm_adjoint_init(g._h, adj_ptr, self.adj_bytes))
        self.dJ.zero_()
        for s0 in reversed(range(0, self.steps, self.K)):
            s1 = min(s0 + self.K, self.steps)
            _restore(g, self.checkpoints[s0])
            g.set_step(s0)
            states: List = []
            for n in range(s0, s1):
                states.append(_snapshot(g))
                g.step(1, rtol=self.rtol, max_iter=self.max_iter, stats=False)
            for n in reversed(range(s0, s1)):
                snap = states[n - s0]
                ptrs = (C.c_void_p * 7)(*[C.c_void_p(t.data_ptr()) for t in snap[:7]])
                g.stream.synchronize()
                bcm._check(L.bcm_adjoint_step(g._h, adj_ptr, self.adj_bytes, ptrs,
                                              1 if n == 0 else 0, 1.0 / self.steps,
                                              self.rtol, self.max_iter,
                                              C.c_void_p(self.dJ.data_ptr())))
        g.stream.synchronize()
        d = self.dJ.cpu().numpy()
        return d[:8].copy(), d[8:].copy()


def _make_function():
    import torch

    class DragFunction(torch.autograd.Function):
        """J(a, c): time-averaged drag; backward by the discrete adjoint."""

        @staticmethod
        def forward(ctx, modes, center, spec, radius, steps, checkpoint_every, rtol):
            run = AdjointRun(spec, modes.detach().cpu().numpy(), center.detach().cpu().numpy(),
                             radius, steps, checkpoint_every, rtol)
            J = run.forward()
            ctx.run = run
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            ga, gc = ctx.run.backward()
            s = float(gJ)
            return (torch.from_numpy(ga * s), torch.from_numpy(gc * s),
                    None, None, None, None, None)

    return DragFunction


def drag(modes, center, spec, radius: float, steps: int, checkpoint_every: int = 10,
         rtol: float = 1e-12):
    """Differentiable time-averaged drag (torch tensors modes[8], center[3], float64)."""
    return _make_function().apply(modes, center, spec, radius, steps, checkpoint_every, rtol)
