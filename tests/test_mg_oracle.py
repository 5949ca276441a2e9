"""Pins of the oracle's multigrid preconditioner (oracle/mg_oracle.py) to things other
than itself: the Galerkin operators of the per-cube levels against the closed form of
the flux-form operator at the coarse spacing (built here from the geometry alone),
symmetry and positive definiteness of M^-1, convergence of the V-cycle as an
iteration, and PCG with M^-1 against a dense direct solve."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg  # noqa: F401  (spsolve)

import oracle as O
from oracle import mg_oracle as MGO
from paper_1808_04099_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def closed_form_level(spec, l):
    """Flux-form operator of a single-sim, single-level grid at level l (cells of
    2^l h): a face between two cells of level l carries 4^l fine faces of coefficient
    h (area h^2 over distance h), so its coefficient is 4^l h; an outflow face (p = 0
    on the face) gives 2 x that on the diagonal, other domain faces nothing, and
    periodic faces wrap."""
    assert spec.n_sims == 1 and spec.max_level == 0
    B = spec.B
    bl = B >> l
    h = spec.sim_h0[0]
    coef = (4.0 ** l) * h
    ext = np.asarray(spec.sim_extent[0]) // (1 << l)
    cubes = np.asarray(spec.cube_ijk).reshape(-1, 3) // B
    index = {}
    n = 0
    for c, cc in enumerate(cubes):
        for k in range(bl):
            for j in range(bl):
                for i in range(bl):
                    index[(cc[0] * bl + i, cc[1] * bl + j, cc[2] * bl + k)] = \
                        (c * bl + k) * bl * bl + j * bl + i
                    n += 1
    rows, cols, vals = [], [], []
    bc = list(spec.sim_bc[0])
    for X, u in index.items():
        diag = 0.0
        for d in range(3):
            for side, step in ((0, -1), (1, 1)):
                Y = list(X)
                Y[d] += step
                f = 2 * d + side
                if 0 <= Y[d] < ext[d]:
                    v = index[tuple(Y)]
                elif bc[f] == W.PERIODIC:
                    Y[d] %= ext[d]
                    v = index[tuple(Y)]
                elif bc[f] == W.OUTFLOW:
                    diag += 2.0 * coef
                    continue
                else:
                    continue
                if v == u:
                    continue
                diag += coef
                rows.append(u)
                cols.append(v)
                vals.append(-coef)
        rows.append(u)
        cols.append(u)
        vals.append(diag)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


GRIDS = {
    "channel": lambda: W.sphere_channel(4, 2, 2, 4, length=(4.0, 2.0, 2.0), radius=0.3),
    "cavity": lambda: W.cavity(2, 4),
    "periodic": lambda: W.periodic_box(2, 4),
}


@pytest.mark.parametrize("name", sorted(GRIDS))
def test_galerkin_levels_equal_closed_form(name):
    spec = GRIDS[name]()
    mg = MGO.MG(O.Oracle(spec))
    L = int(round(math.log2(spec.B)))
    for l in range(L + 1):
        ref = closed_form_level(spec, l)
        diff = abs(mg.Ks[l] - ref).max()
        assert diff <= 1e-12 * abs(ref).max(), (l, diff)


@pytest.mark.parametrize("name", ["channel", "cavity"])
def test_preconditioner_symmetric_positive_definite(name):
    spec = W.sphere_channel(2, 2, 2, 4, length=(2.0, 2.0, 2.0), radius=0.2,
                            center=(0.5, 1.0, 1.0)) if name == "channel" else W.cavity(2, 4)
    mg = MGO.MG(O.Oracle(spec))
    M = mg.matrix()
    assert np.abs(M - M.T).max() <= 1e-13 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0.0


@pytest.mark.parametrize("name", ["cavity", "periodic"])
def test_singular_sims_keep_the_top_correction_at_zero(name):
    """All-Neumann and all-periodic sims: K 1 = 0, so the single top node's Galerkin
    diagonal is zero and its correction is zero; M^-1 stays bounded (no division by the
    round-off of that diagonal) and symmetric."""
    spec = GRIDS[name]()
    mg = MGO.MG(O.Oracle(spec))
    top = mg.Ks[-1].toarray()
    assert top.shape == (1, 1) and abs(top[0, 0]) <= 1e-12 * abs(mg.Ks[0]).max()
    r = np.random.default_rng(5).standard_normal(mg.K.shape[0])
    z = mg.apply(r)
    assert np.linalg.norm(z) <= 10.0 * np.linalg.norm(r / mg.K.diagonal())


def test_preconditioned_spectrum_positive_and_well_conditioned():
    """The eigenvalues of M^-1 K are real and positive (M^-1 SPD), and their spread is
    a small fraction of that of the Jacobi-preconditioned D^-1 K: what CG needs.  (With
    the coarse correction scaled by 1.75 the V-cycle alone is no convergent stationary
    iteration; CG does not need one.)"""
    spec = W.sphere_channel(2, 2, 2, 4, length=(2.0, 2.0, 2.0), radius=0.2,
                            center=(0.5, 1.0, 1.0))
    mg = MGO.MG(O.Oracle(spec))
    K = mg.K.toarray()
    ev = np.linalg.eigvals(mg.matrix() @ K)
    assert np.abs(ev.imag).max() <= 1e-9 * np.abs(ev.real).max()
    ev = ev.real
    assert ev.min() > 0.0
    evj = np.linalg.eigvals(K / np.diag(K)[:, None]).real
    assert ev.max() / ev.min() < 0.1 * evj.max() / evj.min()


def test_mg_pcg_matches_direct_solve_in_fewer_iterations():
    spec = W.sphere_channel(4, 2, 2, 8, radius=0.3)
    mg = MGO.MG(O.Oracle(spec))
    K = mg.K
    b = np.random.default_rng(3).standard_normal(K.shape[0])
    x, it = MGO.pcg(K, b, mg.apply, 1e-11)
    xd = sp.linalg.spsolve(sp.csc_matrix(K), b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    d = K.diagonal()
    _, it_j = MGO.pcg(K, b, lambda r: r / d, 1e-11)
    assert it * 3 < it_j, (it, it_j)


def two_level_small(nx=2, ny=1, nz=1, B=4):
    """A level-0 row of cubes of 4^3 whose first cube is split into eight level-1 cubes
    (2:1 faces in x, and the refined block against the domain walls)."""
    return W.two_level_channel(nx, ny, nz, B, (0, 0, 0), (1, 1, 1), 1.0 / 8.0, 0)


def cell_owner(spec, l):
    """Per level-l cell: its cube and that cube's level."""
    bl = spec.B >> l
    cube = np.repeat(np.arange(spec.n_cubes), bl ** 3)
    return cube, np.asarray(spec.cube_level, np.int64)[cube]


@pytest.mark.parametrize("nx", [2, 3])
def test_two_level_faces_keep_the_21_form_on_every_level(nx):
    """On a two-level grid every per-cube level's Galerkin operator keeps the flux form
    of R7 across a 2:1 face, the form the GPU levels apply: each cell of a coarse cube
    facing the refined block couples to exactly four cells of fine cubes and each fine
    cell on such a face to exactly one coarse cell, with the coefficient of the
    finest level's sub-face scaled by the fine faces it now carries, 4^l h_f / 1.5, and
    same-level faces keep 4^l h of their cube."""
    spec = two_level_small(nx)
    mg = MGO.MG(O.Oracle(spec))
    h0 = spec.sim_h0[0]
    L = int(round(math.log2(spec.B)))
    for l in range(L + 1):
        K = sp.coo_matrix(mg.Ks[l])
        cube, lv = cell_owner(spec, l)
        off = K.row != K.col
        rows, cols, vals = K.row[off], K.col[off], K.data[off]
        cross = lv[rows] != lv[cols]
        assert cross.any()
        want = (4.0 ** l) * (h0 / 2.0) / 1.5
        np.testing.assert_allclose(-vals[cross], want, rtol=1e-12)
        coarse_rows = rows[cross & (lv[rows] == 0)]
        fine_rows = rows[cross & (lv[rows] == 1)]
        assert np.all(np.bincount(coarse_rows)[np.unique(coarse_rows)] == 4)
        assert np.all(np.bincount(fine_rows)[np.unique(fine_rows)] == 1)
        same = ~cross & (cube[rows] != cube[cols])
        hc = h0 / (2.0 ** lv[rows[same]])
        np.testing.assert_allclose(-vals[same], (4.0 ** l) * hc, rtol=1e-12)
        inner = ~cross & (cube[rows] == cube[cols])
        hc = h0 / (2.0 ** lv[rows[inner]])
        np.testing.assert_allclose(-vals[inner], (4.0 ** l) * hc, rtol=1e-12)


def test_two_level_preconditioner_symmetric_positive_definite():
    spec = two_level_small()
    mg = MGO.MG(O.Oracle(spec))
    M = mg.matrix()
    assert np.abs(M - M.T).max() <= 1e-13 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0.0


def test_two_level_mg_pcg_matches_direct_solve_in_fewer_iterations():
    spec = W.two_level_channel(4, 2, 2, 4, (1, 0, 0), (3, 2, 2), 1.0 / 8.0, 0)
    mg = MGO.MG(O.Oracle(spec))
    K = mg.K
    b = np.random.default_rng(4).standard_normal(K.shape[0])
    x, it = MGO.pcg(K, b, mg.apply, 1e-11)
    xd = sp.linalg.spsolve(sp.csc_matrix(K), b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    d = K.diagonal()
    _, it_j = MGO.pcg(K, b, lambda r: r / d, 1e-11)
    assert it * 2 < it_j, (it, it_j)
