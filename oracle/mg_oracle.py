"""Geometric multigrid V-cycle used as the PCG preconditioner M^-1, by its definition.

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` may import this module.  It shares no code
with the CUDA library: the operator is taken from the C oracle (``Oracle.apply_poisson``
on unit vectors), the coarse operators are Galerkin products of sparse matrices, and
every step below is written from its definition with numpy / scipy.

The method's pressure solve (section "Numerical algorithm", Eq. poisson) is a Krylov
solve of K p = -V b; the paper solves it with a geometric multigrid on its cubes.
Here the multigrid is the preconditioner of that CG, on grids of one or two levels:

  levels    per-cube levels l = 0 .. L (L = log2 B): level l has (B / 2^l)^3 cells per
            cube, cell (c, i, j, k) of level l+1 covering cells (c, 2i..2i+1, 2j..2j+1,
            2k..2k+1) of level l; then cube-aggregate levels (level L itself has one
            cell per cube): on a two-level grid first the eight refined cubes of each
            level-0 position join into one node (the other cubes stay as they are),
            then nodes of one sim whose level-0 cube coordinates shifted right by m
            agree form one node, m = 1 .. M, M = max(1, ceil(log2 E)), E the largest
            extent of a sim in level-0 cubes, so every sim ends in one node.
  transfer  P_l: level l+1 -> level l, piecewise constant (each fine unknown takes the
            value of the coarse unknown covering it); restriction P_l^T (sums).
  operators K_0 = K, K_{l+1} = P_l^T K_l P_l (Galerkin).
  smoother  S_l = omega D_l^-1, D_l = diag(K_l) (a zero diagonal gives 0: the top node
            of a sim without outflow faces, where K 1 = 0), omega = 0.8.
  V-cycle   V_l(r):  x = S_l r;  x += s P_l V_{l+1}(P_l^T (r - K_l x));
                     x += S_l (r - K_l x);  return x
            with the coarse correction scaled by s = 1.75: piecewise-constant transfers
            leave the Galerkin correction too weak, and the scale that minimises the
            PCG iteration count on channel, cavity and batched grids is 1.5 - 2
            V_top(r): x = 0; four times x += S (r - K x); return x
  M^-1 r = V_0(r).

The pre- and post-smoothers are the same symmetric S, so M^-1 is symmetric; with
omega < 2 / lambda_max(D^-1 K) (lambda_max <= 2 for these diagonally dominant
operators) its smoother part is positive definite and the scaled coarse part positive
semidefinite, so M^-1 is positive definite for any s > 0.
"""
from __future__ import annotations

import math
from typing import List

import numpy as np
import scipy.sparse as sp

OMEGA = 0.8
NU_TOP = 4
OVER = 1.75  # scale of the coarse-grid correction


def operator_matrix(oracle):
    """K of the oracle's grid, column by column from the oracle's operator (sparse)."""
    n = oracle.n_cells
    rows, cols, vals = [], [], []
    e = np.zeros(n)
    for col in range(n):
        e[col] = 1.0
        k = oracle.apply_poisson(e)
        e[col] = 0.0
        nz = np.nonzero(k)[0]
        rows.append(nz)
        cols.append(np.full(nz.size, col))
        vals.append(k[nz])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def parent_maps(spec) -> List[np.ndarray]:
    """parents[l][u] = the level-(l+1) unknown covering level-l unknown u, for every
    level below the top (per-cube levels, then cube aggregates)."""
    if spec.max_level > 1:
        raise ValueError("the multigrid preconditioner is defined on grids of one or two levels")
    B = spec.B
    L = int(round(math.log2(B)))
    nc = spec.n_cubes
    maps = []
    for l in range(L):
        bl = B >> l
        bc = bl // 2
        par = np.empty(nc * bl ** 3, np.int64)
        for c in range(nc):
            for k in range(bl):
                for j in range(bl):
                    for i in range(bl):
                        par[(c * bl + k) * bl * bl + j * bl + i] = \
                            ((c * bc + k // 2) * bc + j // 2) * bc + i // 2
        maps.append(par)
    # cube aggregates.  cube_ijk are corner coordinates in cells of the finest level, so
    # a cube of level lv spans B 2^(max_level - lv) of them per edge
    sim_of = spec.sim_of_cube()
    lvl = np.asarray(spec.cube_level, np.int64) if spec.max_level else np.zeros(nc, np.int64)
    corner = np.asarray(spec.cube_ijk, np.int64).reshape(-1, 3)
    coords = corner // (B << spec.max_level)  # the level-0 cube position of every cube
    ext = 1
    for s in range(spec.n_sims):
        a, b = spec.sim_cube_offset[s], spec.sim_cube_offset[s + 1]
        cs = coords[a:b]
        ext = max(ext, int((cs.max(axis=0) - cs.min(axis=0) + 1).max()))
    M = max(1, int(math.ceil(math.log2(ext))) if ext > 1 else 1)
    keys = [(int(sim_of[c]),) + tuple(coords[c]) for c in range(nc)]
    node_of = np.arange(nc)
    if spec.max_level:  # the refined cubes of each level-0 position become one node
        newkeys = {}
        par = np.empty(nc, np.int64)
        for c in range(nc):
            key = keys[c] if lvl[c] else keys[c] + (int(c),)
            if key not in newkeys:
                newkeys[key] = len(newkeys)
            par[c] = newkeys[key]
        maps.append(par)
        node_of = par[node_of]
    for m in range(1, M + 1):
        newkeys = {}
        level_keys = {}
        for c in range(nc):
            key = (keys[c][0],) + tuple(x >> m for x in keys[c][1:])
            if key not in newkeys:
                newkeys[key] = len(newkeys)
            level_keys[int(node_of[c])] = newkeys[key]
        par = np.array([level_keys[u] for u in range(len(level_keys))], np.int64)
        maps.append(par)
        node_of = par[node_of]
    return maps


def prolongators(maps: List[np.ndarray]):
    """Piecewise-constant P_l (n_l x n_{l+1}, sparse)."""
    return [sp.csr_matrix((np.ones(par.size), (np.arange(par.size), par)),
                          shape=(par.size, int(par.max()) + 1)) for par in maps]


def galerkin(K, Ps):
    Ks = [sp.csr_matrix(K)]
    for P in Ps:
        Ks.append(sp.csr_matrix(P.T @ Ks[-1] @ P))
    return Ks


def inverse_diagonals(Ks, Ps) -> List[np.ndarray]:
    """omega / diag(K_l) per level; a zero diagonal gives 0.  A Galerkin diagonal is a
    sum of non-negative face coefficients; one that is zero in exact arithmetic (the top
    node of a sim without an outflow face, where K 1 = 0) comes out of the
    floating-point products as round-off, so a diagonal below 1e-12 of the diagonals it
    aggregates (summed in absolute value down to the finest level) counts as zero."""
    mass = np.abs(Ks[0].diagonal())
    out = []
    for l, Kl in enumerate(Ks):
        if l:
            mass = Ps[l - 1].T @ mass
        d = Kl.diagonal()
        zero = np.abs(d) <= 1e-12 * mass
        out.append(np.where(zero, 0.0, OMEGA / np.where(zero, 1.0, d)))
    return out


def vcycle(Ks, Ps, Ws, r: np.ndarray, l: int = 0) -> np.ndarray:
    """V_l(r) as defined in the module docstring (Ws: the smoothers omega D_l^-1)."""
    Kl, S = Ks[l], Ws[l]
    if l == len(Ps):  # top
        x = np.zeros_like(r)
        for _ in range(NU_TOP):
            x = x + S * (r - Kl @ x)
        return x
    P = Ps[l]
    x = S * r
    x = x + OVER * (P @ vcycle(Ks, Ps, Ws, P.T @ (r - Kl @ x), l + 1))
    x = x + S * (r - Kl @ x)
    return x


class MG:
    """The preconditioner of one oracle grid (sparse matrices; small grids: K is built
    from one operator application per cell)."""

    def __init__(self, oracle):
        self.K = operator_matrix(oracle)
        self.maps = parent_maps(oracle.spec)
        self.Ps = prolongators(self.maps)
        self.Ks = galerkin(self.K, self.Ps)
        self.Ws = inverse_diagonals(self.Ks, self.Ps)

    def apply(self, r: np.ndarray) -> np.ndarray:
        return vcycle(self.Ks, self.Ps, self.Ws, np.asarray(r, np.float64))

    def matrix(self) -> np.ndarray:
        """M^-1 as a dense matrix (one V-cycle per column)."""
        n = self.K.shape[0]
        return np.stack([self.apply(np.eye(1, n, i)[0]) for i in range(n)], axis=1)


def pcg(K, b, apply_m, rtol=1e-10, max_iter=10000):
    """Preconditioned CG (Saad, Alg. 9.1) from x = 0; returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    z = apply_m(r)
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    for it in range(max_iter):
        if np.linalg.norm(r) <= rtol * nb:
            return x, it
        q = K @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = apply_m(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_iter
