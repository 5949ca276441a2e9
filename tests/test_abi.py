"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/bcm.h declares; invalid descriptions are rejected on the host."""
import ctypes as C
import os
import re

import numpy as np

from paper_1808_04099_gb300 import bcm, _build
from paper_1808_04099_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(bcm_[a-z_0-9]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    L = C.CDLL(_build.build())
    names = declared()
    assert len(names) >= 10
    for n in sorted(names):
        assert hasattr(L, n), n
    assert names <= set(bcm.EXPORTED)


def test_workspace_bytes_and_invalid_descriptions():
    L = bcm.lib()
    spec = W.sphere_channel(4, 2, 2, 8)

    def desc_for(sp, prec=0, B=None):
        g = bcm.GridDesc()
        arrs = [np.ascontiguousarray(sp.sim_cube_offset, np.int32),
                np.ascontiguousarray(sp.cube_ijk, np.int32),
                np.ascontiguousarray(sp.cube_level, np.int8),
                np.ascontiguousarray(sp.sim_extent, np.int32), sp.sim_origin, sp.sim_h0,
                np.ascontiguousarray(sp.sim_bc, np.int32), sp.sim_bc_vel, sp.sim_nu, sp.sim_dt,
                sp.sim_uconv]
        arrs = [np.ascontiguousarray(a) for a in arrs]
        g.n_sims, g.n_cubes, g.cells_per_edge = sp.n_sims, sp.n_cubes, B or sp.B
        g.max_level, g.precision = sp.max_level, prec
        (g.sim_cube_offset, g.cube_ijk, g.cube_level, g.sim_extent, g.sim_origin, g.sim_h0,
         g.sim_bc, g.sim_bc_vel, g.sim_nu, g.sim_dt, g.sim_uconv) = [a.ctypes.data for a in arrs]
        return g, arrs

    d, keep = desc_for(spec)
    n64 = L.bcm_workspace_bytes(C.byref(d))
    n = spec.n_cells
    assert n64 >= n * 8 * 15   # 13 state/solver fields of 8 bytes + 2 FP64 fields
    d32, keep32 = desc_for(spec, prec=1)
    assert 0 < L.bcm_workspace_bytes(C.byref(d32)) < n64
    dbad, keepb = desc_for(spec, B=5)
    assert L.bcm_workspace_bytes(C.byref(dbad)) == 0
    assert b"cells_per_edge" in L.bcm_last_error()
    hole = W.sphere_channel(4, 2, 2, 8)
    hole.cube_ijk = hole.cube_ijk[:-1].copy()
    hole.cube_level = hole.cube_level[:-1].copy()
    hole.sim_cube_offset = np.array([0, hole.cube_ijk.shape[0]], np.int32)
    dh, keeph = desc_for(hole)
    assert L.bcm_workspace_bytes(C.byref(dh)) == 0
    assert b"no neighbour" in L.bcm_last_error()
    out = C.c_void_p()
    assert L.bcm_create_grid(C.byref(d), None, 0, None, C.byref(out)) == bcm.BCM_E_INVALID
