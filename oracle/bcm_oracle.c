/*
 * bcm_oracle.c -- plain FP64 CPU oracle of the Building Cube Method (BCM) time step.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, by the smoke check and by the
 * CPU-baseline leg of the benchmark, never by the product path.  Deliberately
 * slow and literal: each cube keeps a ghosted (B+4)^3 copy that is refilled by
 * the halo rules before every stencil, and every operator is a nested loop.
 * Reductions are summed per cube in cell order and then over cubes in cube order,
 * so the result does not depend on the number of OpenMP threads.
 *
 * The method, following arXiv:1808.04099:
 *   Grid ("Building Cube Method"): equal cubes of B^3 cells in linear arrays
 *     (corner, level); cell centres x_c + (i+1/2)h (Eq. cell-center); halo cells
 *     filled by copying the neighbour's boundary interior cells (same level),
 *     by a weighted mean of fine cells (fine -> coarse) and by copying the coarse
 *     cell into every fine halo cell it covers (coarse -> fine).
 *   Step ("Numerical algorithm", Eq. substep1, Eq. poisson):
 *     1. momentum sub-step without the body force -> u~
 *     2. IB forcing u* = u~ + (dt/rho) P[F], F = (rho/dt)(U_s - I[u~])
 *     3. pressure Poisson D p = (rho/dt) G.u*
 *     4. projection u^{n+1} = u* - (dt/rho) G p
 *
 * Readings where the paper is silent, garbled or at odds with itself:
 *   R1 projection prefactor: the printed correction carries rho/dt, which is
 *      dimensionally inconsistent with Eq. poisson; dt/rho is used so that the
 *      corrected face velocities are discretely divergence free.
 *   R2 collocated projection: divergence and pressure gradients act on face
 *      velocities U_f = (u_i + u_nb)/2; the cell velocity receives the mean of its
 *      two face gradients per axis (approximate projection).
 *   R3 time scheme: explicit, the convection by 2nd-order Adams-Bashforth and the
 *      diffusion by forward Euler; the first step uses N^{-1} := N^0.
 *   R4 dt = min(0.3 h/U, h^2/(8 nu)) (chosen by the workload, passed in).
 *   R5 IB with a per-cell solid fraction phi = (1 - tanh(d/eps))/2, eps = 1.5 h,
 *      d the signed distance (phi = 0 where d >= 20 eps); u* = u~ + phi (u_s - u~),
 *      i.e. the interpolation/spreading pair collapses to the cell itself.
 *   R6 fine -> coarse halo weights w = 1/8 (mean of the 2x2x2 fine cells).
 *   R7 the Poisson operator at 2:1 faces is flux form (sub-face area h_f^2,
 *      distance 0.75 h_c) so that K = -V A stays symmetric for CG; momentum
 *      uses the paper's halo values with the cube's own stencil.
 *   R8 boundary conditions: WALL / INFLOW velocity ghosts 2 w - u_0; SLIP mirror
 *      (normal component negated); OUTFLOW: ghosts 2 u_b - u_0 with the face value
 *      u_b advected by du_b/dt + U_c (u_b - u_0)/(h/2) = 0; pressure Neumann
 *      except p = 0 at OUTFLOW faces; PERIODIC by adjacency.
 *   R9 ellipsoid signed distance d ~ k0 (k0 - 1) / k1, k0 = |y/a|, k1 = |y/a^2|.
 *   R10 all-Neumann sims: the volume mean of b is removed before the solve.
 *   R11 Jacobi-preconditioned CG (Saad, Alg. 9.1) on K p = -V b, warm start p^n,
 *      stop when the recurrence residual ||r|| <= rtol ||-V b||.
 *   R19 Lagrangian particles (orc_step_particles; section "Lagrangian-Eulerian
 *      Interaction", Eqs. ddeltai and ddeltap, the forcing sub-step and the position
 *      update of "Numerical algorithm"), on single-level grids: the 27 cells whose
 *      centres lie within 1.5 h of a particle per axis carry the weights
 *      phi(r_x) phi(r_y) phi(r_z) of the smoothed 3-point delta; cells outside the
 *      domain are left out of both sums (no wrap at periodic faces).  U_s^n is the
 *      velocity of the particle's body at (X^n, t^n); the position update takes the
 *      body velocity at (X^n, t^{n+1}).  rho = 1; the force on the body is
 *      -sum_p F_p dV_p.  The solid fraction is zero in this mode.
 *   R20 QUICK + Crank-Nicolson momentum (orc_set_scheme; Eq. substep1 with the QUICK
 *      scheme the paper names for its convection): convective face values by
 *      quadratic upstream interpolation phi_f = 6/8 phi_C + 3/8 phi_D - 1/8 phi_U (C the
 *      upwind cell, D the downwind one, U the cell upwind of C) on the central face
 *      velocities; diffusion the 7-point Laplacian.  The implicit half is solved by the
 *      iteration from the forward-Euler predictor u^(0) = 2 E - u^n,
 *        u^(k+1) = (E - dt/2 N(u^(k)) + dt nu/2 (sum of the 6 neighbours of u^(k))/h^2)
 *                  / (1 + 3 dt nu / h^2),     E = u^n + dt (-N(u^n)/2 + nu L(u^n)/2),
 *      whose fixed point is the Crank-Nicolson step; E takes the ghosts of u^n (outflow
 *      face values of t^n), and the ghosts of u^(k), iterates of u~ and so velocities of
 *      t^{n+1}, follow the halo rules with the outflow face values of t^{n+1} (R8's update
 *      from u^n).  The start u^(0) and the two stops below move the result by no more
 *      than the iteration tolerance: the fixed point is unique.  A sim stops iterating once
 *      ||u^(k+1) - u^(k)|| <= cn_rtol ||u^(k+1)|| (all three components), once the update
 *      has reached the rounding floor of the arithmetic (at most 64 eps ||u^(k+1)||, eps
 *      the unit roundoff) and no longer shrinks (its square >= 0.99 of the previous
 *      one), or after cn_max iterations.  The IB forcing then acts on the result.
 *   R21 wavelet compression of a field (orc_wavelet_*; section "Data compression"): per
 *      cube, L = log2 B levels of a separable 3-D CDF 5/3 lifting transform of the B^3
 *      interior values (the paper cites Sakai et al. for its wavelet without printing
 *      it; the halo is not transformed: a restart rebuilds it from the neighbours):
 *        d_i = x_{2i+1} - (x_{2i} + x_{2i+2})/2,  s_i = x_{2i} + (d_{i-1} + d_i)/4,
 *      symmetric at the ends (x_{2h} := x_{2h-2}, d_{-1} := d_0), passes x, y, z per
 *      level on the low band, coefficients kept in place (s first, then d along each
 *      line).  One uniform quantizer q = rint(c / step); a Golomb-Rice coder replaces
 *      zlib: z = zigzag(q), k = floor(log2(mean z)) per cube (0 if the mean is 0, at most
 *      24); u = z >> k below 16 is written as u one-bits, a zero-bit and the k low bits of
 *      z, else as 16 one-bits and the 32 bits of z; bits LSB-first in 32-bit words.
 *      Stream of 32-bit words: magic, version, B, n_cubes, 0, 0, step (2 words), the
 *      word count of every cube record, then the records: a word k | nbits << 5 and the
 *      ceil(nbits / 32) payload words.  All arithmetic in FP64 without contraction.
 */
#include "bcm_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define H 2
#define NB_BOUNDARY (-1)
#define NB_COARSE (-2)
#define NB_FINE (-3)

enum { BC_WALL = 0, BC_INFLOW = 1, BC_SLIP = 2, BC_OUTFLOW = 3, BC_PERIODIC = 4 };
enum { BODY_NONE = 0, BODY_SPHERE = 1, BODY_ELLIPSOID = 2 };

static const int mode_k[ORC_NMODES] = {1, 1, 2, 2, 1, 3, 2, 3};
static const int mode_l[ORC_NMODES] = {1, 2, 1, 2, 3, 1, 3, 2};

static char g_err[256];
const char *orc_error(void) { return g_err; }

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops from now on (n >= 1); returns the previous count.
 * Results do not depend on it: per-cube partial sums are added in cube order. */
int orc_set_threads(int n) {
    const int old = orc_threads();
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
    return old;
}

struct orc_grid {
    int B, G, max_level, n_sims, n_cubes, n_slots;
    int32_t *sim_off, *ijk, *extent, *bc, *sim_of, *level;
    double *origin, *h0, *bcvel, *nu, *dt, *uconv, *bodies, *modes;
    int32_t *nb;        /* [c*6+f] */
    int32_t *nb_coarse; /* [c*6+f] coarse cube id when nb == NB_COARSE */
    int32_t *nb_fine;   /* [(c*6+f)*4 + qb*2 + qa] when nb == NB_FINE */
    int32_t *slot;      /* [c*6+f] outflow slot or -1 */
    int32_t *order;     /* cube ids sorted by (sim, level, z, y, x) */
    int scheme;         /* momentum: 0 AB2 + central, 1 QUICK + Crank-Nicolson (R20) */
    double cn_rtol;     /* Crank-Nicolson iteration: relative update per sim */
    int cn_max;         /*   and the most iterations per step */
    int ab2_restart;    /* the next AB2 step takes N^{n-1} := N^n (after Crank-Nicolson) */
};

/* ------------------------------------------------------------------ helpers */

static int tan1(int d) { return d == 0 ? 1 : 0; }
static int tan2(int d) { return d == 2 ? 1 : 2; }
static int cell_span(const orc_grid *g, int c) { return 1 << (g->max_level - g->level[c]); }
static double cell_h(const orc_grid *g, int c) {
    return g->h0[g->sim_of[c]] / (double)(1 << g->level[c]);
}
static size_t gidx(const orc_grid *g, int i, int j, int k) {
    return ((size_t)(k + H) * g->G + (size_t)(j + H)) * g->G + (size_t)(i + H);
}
static size_t cidx(int B, int c, int i, int j, int k) {
    return (size_t)c * B * B * B + ((size_t)k * B + j) * B + i;
}
/* interior index of a cell given normal axis d, normal index n and tangential (a, b) */
static void put_ijk(int d, int n, int a, int b, int *ijk) {
    ijk[d] = n;
    ijk[tan1(d)] = a;
    ijk[tan2(d)] = b;
}

/* cube lookup by binary search over cubes sorted by (sim, level, z, y, x) */
static const orc_grid *g_sort_grid;
static int key_cmp4(const int32_t *a, const int32_t *b) {
    for (int e = 0; e < 5; ++e)
        if (a[e] != b[e]) return a[e] < b[e] ? -1 : 1;
    return 0;
}
static void cube_key(const orc_grid *g, int c, int32_t *key) {
    key[0] = g->sim_of[c];
    key[1] = g->level[c];
    key[2] = g->ijk[3 * c + 2];
    key[3] = g->ijk[3 * c + 1];
    key[4] = g->ijk[3 * c];
}
static int sort_cmp(const void *pa, const void *pb) {
    int32_t ka[5], kb[5];
    cube_key(g_sort_grid, *(const int32_t *)pa, ka);
    cube_key(g_sort_grid, *(const int32_t *)pb, kb);
    return key_cmp4(ka, kb);
}
static int find_cube(const orc_grid *g, int s, int lev, int x, int y, int z) {
    int32_t want[5] = {s, lev, z, y, x};
    int lo = 0, hi = g->n_cubes - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        int32_t key[5];
        cube_key(g, g->order[mid], key);
        int cmp = key_cmp4(key, want);
        if (cmp == 0) return g->order[mid];
        if (cmp < 0) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

static int wrap(int x, int n) { return ((x % n) + n) % n; }

/* -------------------------------------------------------------- grid build */

orc_grid *orc_create(int B, int max_level, int n_sims, int n_cubes, const int32_t *sim_off,
                     const int32_t *ijk, const int8_t *level, const int32_t *extent,
                     const double *origin, const double *h0, const int32_t *bc,
                     const double *bcvel, const double *nu, const double *dt,
                     const double *uconv, const double *bodies, const double *modes) {
    orc_grid *g = (orc_grid *)calloc(1, sizeof(orc_grid));
    g->B = B;
    g->G = B + 2 * H;
    g->max_level = max_level;
    g->n_sims = n_sims;
    g->n_cubes = n_cubes;
#define DUP(dst, src, n, T)                                 \
    do {                                                    \
        dst = (T *)malloc(sizeof(T) * (size_t)(n) + 1);     \
        memcpy(dst, src, sizeof(T) * (size_t)(n));          \
    } while (0)
    DUP(g->sim_off, sim_off, n_sims + 1, int32_t);
    DUP(g->ijk, ijk, 3 * n_cubes, int32_t);
    DUP(g->extent, extent, 3 * n_sims, int32_t);
    DUP(g->bc, bc, 6 * n_sims, int32_t);
    DUP(g->origin, origin, 3 * n_sims, double);
    DUP(g->h0, h0, n_sims, double);
    DUP(g->bcvel, bcvel, 18 * n_sims, double);
    DUP(g->nu, nu, n_sims, double);
    DUP(g->dt, dt, n_sims, double);
    DUP(g->uconv, uconv, n_sims, double);
    DUP(g->bodies, bodies, n_sims * ORC_MAX_BODIES * ORC_BODY_STRIDE, double);
    DUP(g->modes, modes, n_sims * ORC_NMODES, double);
#undef DUP
    g->level = (int32_t *)malloc(sizeof(int32_t) * n_cubes + 1);
    g->sim_of = (int32_t *)malloc(sizeof(int32_t) * n_cubes + 1);
    for (int c = 0; c < n_cubes; ++c) g->level[c] = level[c];
    for (int s = 0; s < n_sims; ++s)
        for (int c = sim_off[s]; c < sim_off[s + 1]; ++c) g->sim_of[c] = s;
    g->nb = (int32_t *)malloc(sizeof(int32_t) * 6 * n_cubes + 1);
    g->nb_coarse = (int32_t *)malloc(sizeof(int32_t) * 6 * n_cubes + 1);
    g->nb_fine = (int32_t *)malloc(sizeof(int32_t) * 24 * n_cubes + 1);
    g->slot = (int32_t *)malloc(sizeof(int32_t) * 6 * n_cubes + 1);
    g->order = (int32_t *)malloc(sizeof(int32_t) * n_cubes + 1);
    for (int c = 0; c < n_cubes; ++c) g->order[c] = c;
    g->scheme = 0;
    g->cn_rtol = 1e-10;
    g->cn_max = 100;
    g->ab2_restart = 0;
    g_sort_grid = g;
    qsort(g->order, (size_t)n_cubes, sizeof(int32_t), sort_cmp);
    for (int c = 1; c < n_cubes; ++c) {
        int32_t ka[5], kb[5];
        cube_key(g, g->order[c - 1], ka);
        cube_key(g, g->order[c], kb);
        if (key_cmp4(ka, kb) == 0) {
            snprintf(g_err, sizeof g_err, "duplicate cube %d", g->order[c]);
            free(g->nb); free(g->nb_coarse); free(g->nb_fine); free(g->slot);
            g->nb = g->nb_coarse = g->nb_fine = g->slot = NULL;
            orc_destroy(g);
            return NULL;
        }
    }

    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : bad)
    for (int c = 0; c < n_cubes; ++c) {
        int s = g->sim_of[c], lev = g->level[c];
        int sp = B * cell_span(g, c);
        const int *ext = &g->extent[3 * s];
        for (int f = 0; f < 6; ++f) {
            int d = f / 2, side = f % 2, bcf = g->bc[6 * s + f];
            int X[3] = {g->ijk[3 * c], g->ijk[3 * c + 1], g->ijk[3 * c + 2]};
            int on_edge = side ? (X[d] + sp == ext[d]) : (X[d] == 0);
            g->nb[6 * c + f] = -100;
            g->nb_coarse[6 * c + f] = -1;
            for (int q = 0; q < 4; ++q) g->nb_fine[(6 * c + f) * 4 + q] = -1;
            if (on_edge && bcf != BC_PERIODIC) {
                g->nb[6 * c + f] = NB_BOUNDARY;
                continue;
            }
            /* same level */
            int Y[3] = {X[0], X[1], X[2]};
            Y[d] = wrap(X[d] + (side ? sp : -sp), ext[d]);
            int n = find_cube(g, s, lev, Y[0], Y[1], Y[2]);
            if (n >= 0) {
                g->nb[6 * c + f] = n;
                continue;
            }
            /* coarser: the cube containing the first point outside the face */
            if (lev > 0) {
                int csp = 2 * sp, P[3] = {X[0], X[1], X[2]};
                P[d] = wrap(X[d] + (side ? sp : -1), ext[d]);
                int Q[3];
                for (int e = 0; e < 3; ++e) Q[e] = (P[e] / csp) * csp;
                n = find_cube(g, s, lev - 1, Q[0], Q[1], Q[2]);
                if (n >= 0) {
                    g->nb[6 * c + f] = NB_COARSE;
                    g->nb_coarse[6 * c + f] = n;
                    continue;
                }
            }
            /* finer: four cubes of half the span across the face */
            if (lev < g->max_level) {
                int fsp = sp / 2, ok = 1;
                for (int qb = 0; qb < 2; ++qb)
                    for (int qa = 0; qa < 2; ++qa) {
                        int Z[3] = {X[0], X[1], X[2]};
                        Z[d] = wrap(X[d] + (side ? sp : -fsp), ext[d]);
                        Z[tan1(d)] += qa * fsp;
                        Z[tan2(d)] += qb * fsp;
                        int m = find_cube(g, s, lev + 1, Z[0], Z[1], Z[2]);
                        g->nb_fine[(6 * c + f) * 4 + qb * 2 + qa] = m;
                        if (m < 0) ok = 0;
                    }
                if (ok) {
                    g->nb[6 * c + f] = NB_FINE;
                    continue;
                }
            }
            bad += 1;
        }
    }
    if (bad) {
        snprintf(g_err, sizeof g_err, "grid has %d cube faces without a neighbour", bad);
        orc_destroy(g);
        return NULL;
    }
    int k = 0;
    for (int c = 0; c < n_cubes; ++c)
        for (int f = 0; f < 6; ++f)
            g->slot[6 * c + f] =
                (g->nb[6 * c + f] == NB_BOUNDARY && g->bc[6 * g->sim_of[c] + f] == BC_OUTFLOW)
                    ? k++
                    : -1;
    g->n_slots = k;
    return g;
}

void orc_destroy(orc_grid *g) {
    if (!g) return;
    free(g->sim_off); free(g->ijk); free(g->extent); free(g->bc); free(g->origin);
    free(g->h0); free(g->bcvel); free(g->nu); free(g->dt); free(g->uconv); free(g->bodies);
    free(g->modes); free(g->level); free(g->sim_of); free(g->nb); free(g->nb_coarse);
    free(g->nb_fine); free(g->slot); free(g->order);
    free(g);
}

int orc_n_slots(const orc_grid *g) { return g->n_slots; }

void orc_neighbors(const orc_grid *g, int32_t *out) {
    memcpy(out, g->nb, sizeof(int32_t) * 6 * (size_t)g->n_cubes);
}

/* ------------------------------------------------- boundary velocity values */

/* physical centre coordinate of cell index n (may be a halo index) along axis e */
static double centre(const orc_grid *g, int c, int e, int n) {
    int s = g->sim_of[c];
    double hf = g->h0[s] / (double)(1 << g->max_level);
    return g->origin[3 * s + e] + g->ijk[3 * c + e] * hf + (n + 0.5) * cell_h(g, c);
}

/* wall / inflow velocity component `comp` on face f of cube c at tangential cell (a, b) */
static double face_velocity(const orc_grid *g, int c, int f, int comp, int a, int b) {
    int s = g->sim_of[c], d = f / 2;
    double w = g->bcvel[18 * s + 3 * f + comp];
    if (g->bc[6 * s + f] == BC_INFLOW) {
        double hf = g->h0[s] / (double)(1 << g->max_level);
        int e1 = tan1(d), e2 = tan2(d);
        double L1 = g->extent[3 * s + e1] * hf, L2 = g->extent[3 * s + e2] * hf;
        double y = centre(g, c, e1, a) - g->origin[3 * s + e1];
        double z = centre(g, c, e2, b) - g->origin[3 * s + e2];
        double prof = 1.0;
        for (int m = 0; m < ORC_NMODES; ++m)
            prof += g->modes[ORC_NMODES * s + m] * sin(mode_k[m] * M_PI * y / L1) *
                    sin(mode_l[m] * M_PI * z / L2);
        w *= prof;
    }
    return w;
}

/* --------------------------------------------------------------- ghost fill */

static double fval(const orc_grid *g, const double *f, int c, int d, int n, int a, int b) {
    int q[3];
    put_ijk(d, n, a, b, q);
    return f[cidx(g->B, c, q[0], q[1], q[2])];
}

/* Fill the face halos (2 layers) of cube c into its ghosted buffer gb. */
static void fill_cube(const orc_grid *g, const double *f, int kind, const double *ub, int c,
                      double *gb) {
    int B = g->B, s = g->sim_of[c];
    memset(gb, 0, sizeof(double) * (size_t)g->G * g->G * g->G);
    for (int k = 0; k < B; ++k)
        for (int j = 0; j < B; ++j)
            for (int i = 0; i < B; ++i) gb[gidx(g, i, j, k)] = f[cidx(B, c, i, j, k)];
    for (int fc = 0; fc < 6; ++fc) {
        int d = fc / 2, side = fc % 2, nb = g->nb[6 * c + fc];
        for (int layer = 0; layer < H; ++layer) {
            int ng = side ? B + layer : -1 - layer;  /* halo index along d */
            int mirror = side ? B - 1 - layer : layer;
            for (int b = 0; b < B; ++b)
                for (int a = 0; a < B; ++a) {
                    double val = 0.0;
                    if (nb >= 0) {
                        val = fval(g, f, nb, d, side ? layer : B - 1 - layer, a, b);
                    } else if (nb == NB_COARSE) {
                        int C = g->nb_coarse[6 * c + fc];
                        int sf = cell_span(g, c), sc = cell_span(g, C);
                        int A = (g->ijk[3 * c + tan1(d)] + a * sf - g->ijk[3 * C + tan1(d)]) / sc;
                        int Bb = (g->ijk[3 * c + tan2(d)] + b * sf - g->ijk[3 * C + tan2(d)]) / sc;
                        val = fval(g, f, C, d, side ? 0 : B - 1, A, Bb);
                    } else if (nb == NB_FINE) {
                        int qa = (2 * a) / B, qb = (2 * b) / B;
                        int F = g->nb_fine[(6 * c + fc) * 4 + qb * 2 + qa];
                        int fa = 2 * a - qa * B, fb = 2 * b - qb * B;
                        double sum = 0.0;
                        for (int l2 = 0; l2 < 2; ++l2) {
                            int fn = side ? 2 * layer + l2 : B - 1 - 2 * layer - l2;
                            for (int bb = 0; bb < 2; ++bb)
                                for (int aa = 0; aa < 2; ++aa)
                                    sum += fval(g, f, F, d, fn, fa + aa, fb + bb);
                        }
                        val = 0.125 * sum;
                    } else { /* domain boundary */
                        int bcf = g->bc[6 * s + fc];
                        double u0 = fval(g, f, c, d, mirror, a, b);
                        if (kind == 3) {
                            val = (bcf == BC_OUTFLOW) ? -u0 : u0;
                        } else if (bcf == BC_SLIP) {
                            val = (kind == d) ? -u0 : u0;
                        } else if (bcf == BC_OUTFLOW) {
                            int sl = g->slot[6 * c + fc];
                            double vb = ub[(((size_t)sl * 3 + kind) * B + b) * B + a];
                            val = 2.0 * vb - u0;
                        } else { /* WALL, INFLOW */
                            val = 2.0 * face_velocity(g, c, fc, kind, a, b) - u0;
                        }
                    }
                    int q[3];
                    put_ijk(d, ng, a, b, q);
                    gb[gidx(g, q[0], q[1], q[2])] = val;
                }
        }
    }
}

void orc_fill_ghosts(const orc_grid *g, const double *f, int kind, const double *ub,
                     double *out) {
    size_t G3 = (size_t)g->G * g->G * g->G;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < g->n_cubes; ++c) fill_cube(g, f, kind, ub, c, out + (size_t)c * G3);
}

/* ------------------------------------------------------------ solid bodies */

/* rotation matrix of the unit quaternion (w, x, y, z) */
static void quat_mat(const double *q, double R[3][3]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

/* Rodrigues rotation by the vector theta (angle |theta| about theta/|theta|) */
static void rot_vec(const double *th, double R[3][3]) {
    double a = sqrt(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
    if (a == 0.0) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) R[i][j] = (i == j);
        return;
    }
    double k[3] = {th[0] / a, th[1] / a, th[2] / a}, c = cos(a), s = sin(a);
    double K[3][3] = {{0, -k[2], k[1]}, {k[2], 0, -k[0]}, {-k[1], k[0], 0}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double kk = 0;
            for (int m = 0; m < 3; ++m) kk += K[i][m] * K[m][j];
            R[i][j] = (i == j) + s * K[i][j] + (1 - c) * kk;
        }
}

/* Signed distance of point x to body b of sim s at time t, and body velocity there.
 * The body moves rigidly: centre c0 + v t, orientation exp(t [omega]x) R0. */
static double body_sd(const double *body, double t, const double *x, double *vel) {
    int kind = (int)body[0];
    const double *c0 = body + 1, *ax = body + 4, *q = body + 7, *om = body + 11, *v = body + 14;
    double c[3], r[3];
    for (int e = 0; e < 3; ++e) {
        c[e] = c0[e] + v[e] * t;
        r[e] = x[e] - c[e];
    }
    vel[0] = v[0] + om[1] * r[2] - om[2] * r[1];
    vel[1] = v[1] + om[2] * r[0] - om[0] * r[2];
    vel[2] = v[2] + om[0] * r[1] - om[1] * r[0];
    if (kind == BODY_SPHERE) return sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) - ax[0];
    double R0[3][3], Rt[3][3], R[3][3], th[3] = {om[0] * t, om[1] * t, om[2] * t};
    quat_mat(q, R0);
    rot_vec(th, Rt);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            R[i][j] = 0;
            for (int m = 0; m < 3; ++m) R[i][j] += Rt[i][m] * R0[m][j];
        }
    double y[3]; /* body frame: y = R^T r */
    for (int j = 0; j < 3; ++j) y[j] = R[0][j] * r[0] + R[1][j] * r[1] + R[2][j] * r[2];
    double k0 = 0, k1 = 0;
    for (int e = 0; e < 3; ++e) {
        k0 += (y[e] / ax[e]) * (y[e] / ax[e]);
        k1 += (y[e] / (ax[e] * ax[e])) * (y[e] / (ax[e] * ax[e]));
    }
    k0 = sqrt(k0);
    k1 = sqrt(k1);
    if (k1 == 0.0) {
        double m = ax[0];
        if (ax[1] < m) m = ax[1];
        if (ax[2] < m) m = ax[2];
        return -m;
    }
    return k0 * (k0 - 1.0) / k1;
}

/* phi and u_s of one cell: nearest body by signed distance */
static double cell_phi(const orc_grid *g, int c, int i, int j, int k, double t, double *usv) {
    int s = g->sim_of[c];
    double x[3] = {centre(g, c, 0, i), centre(g, c, 1, j), centre(g, c, 2, k)};
    double best = INFINITY;
    usv[0] = usv[1] = usv[2] = 0.0;
    for (int b = 0; b < ORC_MAX_BODIES; ++b) {
        const double *body = g->bodies + ((size_t)s * ORC_MAX_BODIES + b) * ORC_BODY_STRIDE;
        if ((int)body[0] == BODY_NONE) continue;
        double vel[3];
        double d = body_sd(body, t, x, vel);
        if (d < best) {
            best = d;
            usv[0] = vel[0]; usv[1] = vel[1]; usv[2] = vel[2];
        }
    }
    double eps = 1.5 * cell_h(g, c);
    if (!(best < 20.0 * eps)) return 0.0;
    return 0.5 * (1.0 - tanh(best / eps));
}

void orc_solid_fraction(const orc_grid *g, const double *t, double *phi, double *us,
                        double *vs, double *ws) {
    int B = g->B;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < g->n_cubes; ++c)
        for (int k = 0; k < B; ++k)
            for (int j = 0; j < B; ++j)
                for (int i = 0; i < B; ++i) {
                    double v3[3];
                    size_t id = cidx(B, c, i, j, k);
                    phi[id] = cell_phi(g, c, i, j, k, t[g->sim_of[c]], v3);
                    if (us) { us[id] = v3[0]; vs[id] = v3[1]; ws[id] = v3[2]; }
                }
}

/* ------------------------------------------------ Lagrangian particles (R19) */

/* One-dimensional smoothed 3-point delta phi(r) (section "Lagrangian-Eulerian
 * Interaction", the function printed after Eq. ddeltap). */
double orc_delta3(double r) {
    double a = fabs(r);
    if (a <= 0.5) return 0.75 - r * r;
    if (a <= 1.5) return 0.5 * (2.25 - 3.0 * a + r * r);
    return 0.0;
}

/* Index of level-0 cell (I, J, K) of sim s (cells counted from the sim origin), or -1
 * outside the domain or where no cube covers it. */
static long particle_cell(const orc_grid *g, int s, int I, int J, int K) {
    const int *ext = &g->extent[3 * s];
    int B = g->B;
    if (I < 0 || J < 0 || K < 0 || I >= ext[0] || J >= ext[1] || K >= ext[2]) return -1;
    int c = find_cube(g, s, 0, I - I % B, J - J % B, K - K % B);
    if (c < 0) return -1;
    return (long)cidx(B, c, I % B, J % B, K % B);
}

/* The 27 cells around particle X of sim s and their delta weights (product of the
 * three 1-D weights, which already carry the h^3 of Eq. ddeltai).  Returns the count;
 * cells outside the domain are dropped. */
static int particle_stencil(const orc_grid *g, int s, const double *X, long *cell, double *wt) {
    double h = g->h0[s];
    int n = 0;
    int ic[3];
    double xi[3];
    for (int e = 0; e < 3; ++e) {
        xi[e] = (X[e] - g->origin[3 * s + e]) / h;
        ic[e] = (int)floor(xi[e]);
    }
    for (int dk = -1; dk <= 1; ++dk)
        for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
                int I = ic[0] + di, J = ic[1] + dj, K = ic[2] + dk;
                double w = orc_delta3(I + 0.5 - xi[0]) * orc_delta3(J + 0.5 - xi[1]) *
                           orc_delta3(K + 0.5 - xi[2]);
                long id = particle_cell(g, s, I, J, K);
                if (id < 0) continue;
                cell[n] = id;
                wt[n] = w;
                ++n;
            }
    return n;
}

void orc_ib_interpolate(const orc_grid *g, const double *f, int n, const double *X,
                        const int32_t *psim, double *out) {
    for (int q = 0; q < n; ++q) {
        long cell[27];
        double wt[27], U = 0.0;
        int m = particle_stencil(g, psim[q], X + 3 * q, cell, wt);
        for (int a = 0; a < m; ++a) U += f[cell[a]] * wt[a];
        out[q] = U;
    }
}

void orc_ib_spread(const orc_grid *g, int n, const double *X, const int32_t *psim,
                   const double *F, const double *dV, double *out) {
    for (int q = 0; q < n; ++q) {
        long cell[27];
        double wt[27];
        int s = psim[q];
        double h = g->h0[s];
        int m = particle_stencil(g, s, X + 3 * q, cell, wt);
        for (int a = 0; a < m; ++a) out[cell[a]] += F[q] * wt[a] * (dV[q] / (h * h * h));
    }
}

/* Body velocity of particle q at time t (the rigid motion of its body). */
static void particle_body_velocity(const orc_grid *g, int s, int b, const double *X, double t,
                                   double *vel) {
    const double *body = g->bodies + ((size_t)s * ORC_MAX_BODIES + b) * ORC_BODY_STRIDE;
    if ((int)body[0] == BODY_NONE) {
        vel[0] = vel[1] = vel[2] = 0.0;
        return;
    }
    (void)body_sd(body, t, X, vel);
}

void orc_ib_body_velocity(const orc_grid *g, int n, const double *X, const int32_t *psim,
                          const int32_t *pbody, const double *t, double *vel) {
    for (int q = 0; q < n; ++q)
        particle_body_velocity(g, psim[q], pbody[q], X + 3 * q, t[psim[q]], vel + 3 * q);
}

/* ------------------------------------------------------ momentum operators */

/* Conservative central convection N_comp and Laplacian of component comp at (i,j,k),
 * from ghosted velocity buffers gu[3] of one cube with cell size h. */
static void conv_diff(const orc_grid *g, double *const gu[3], int comp, int i, int j, int k,
                      double h, double *Nout, double *Lout) {
    int q[3] = {i, j, k};
    double N = 0.0, L = 0.0;
    const double *uc = gu[comp];
    double u0 = uc[gidx(g, i, j, k)];
    for (int d = 0; d < 3; ++d) {
        int p[3] = {q[0], q[1], q[2]}, m[3] = {q[0], q[1], q[2]};
        p[d] += 1;
        m[d] -= 1;
        size_t ip = gidx(g, p[0], p[1], p[2]), im = gidx(g, m[0], m[1], m[2]),
               i0 = gidx(g, i, j, k);
        const double *ud = gu[d];
        double Fp = 0.5 * (ud[i0] + ud[ip]) * 0.5 * (u0 + uc[ip]);
        double Fm = 0.5 * (ud[im] + ud[i0]) * 0.5 * (uc[im] + u0);
        N += Fp - Fm;
        L += uc[ip] - 2.0 * u0 + uc[im];
    }
    *Nout = N / h;
    *Lout = L / (h * h);
}

/* QUICK face value from the upwind cell C, the downwind cell D and the cell U upwind of
 * C (R20). */
static double quick_face(double pC, double pD, double pU) {
    return 0.75 * pC + 0.375 * pD - 0.125 * pU;
}

/* QUICK convection N_comp at (i,j,k) of a ghosted cube: (1/h) sum_d of the face
 * velocity (central) times the QUICK value of component comp, + face minus - face. */
static double conv_quick(const orc_grid *g, double *const gu[3], int comp, int i, int j,
                         int k, double h) {
    const double *uc = gu[comp];
    size_t i0 = gidx(g, i, j, k);
    double N = 0.0;
    for (int d = 0; d < 3; ++d) {
        int q1[3] = {i, j, k}, q2[3] = {i, j, k}, m1[3] = {i, j, k}, m2[3] = {i, j, k};
        q1[d] += 1; q2[d] += 2; m1[d] -= 1; m2[d] -= 2;
        size_t ip = gidx(g, q1[0], q1[1], q1[2]), ip2 = gidx(g, q2[0], q2[1], q2[2]);
        size_t im = gidx(g, m1[0], m1[1], m1[2]), im2 = gidx(g, m2[0], m2[1], m2[2]);
        const double *ud = gu[d];
        double Up = 0.5 * (ud[i0] + ud[ip]), Um = 0.5 * (ud[im] + ud[i0]);
        double fp = Up >= 0.0 ? quick_face(uc[i0], uc[ip], uc[im])
                              : quick_face(uc[ip], uc[i0], uc[ip2]);
        double fm = Um >= 0.0 ? quick_face(uc[im], uc[i0], uc[im2])
                              : quick_face(uc[i0], uc[im], uc[ip]);
        N += Up * fp - Um * fm;
    }
    return N / h;
}

/* QUICK convection of every component (test path, like orc_convection_diffusion). */
void orc_convection_quick(const orc_grid *g, const double *u, const double *v, const double *w,
                          const double *ub, double *nx, double *ny, double *nz) {
    int B = g->B;
    size_t G3 = (size_t)g->G * g->G * g->G;
    double *gu = (double *)malloc(sizeof(double) * G3 * g->n_cubes);
    double *gv = (double *)malloc(sizeof(double) * G3 * g->n_cubes);
    double *gw = (double *)malloc(sizeof(double) * G3 * g->n_cubes);
    orc_fill_ghosts(g, u, 0, ub, gu);
    orc_fill_ghosts(g, v, 1, ub, gv);
    orc_fill_ghosts(g, w, 2, ub, gw);
    double *No[3] = {nx, ny, nz};
#pragma omp parallel for schedule(static)
    for (int c = 0; c < g->n_cubes; ++c) {
        double *bufs[3] = {gu + c * G3, gv + c * G3, gw + c * G3};
        double h = cell_h(g, c);
        for (int k = 0; k < B; ++k)
            for (int j = 0; j < B; ++j)
                for (int i = 0; i < B; ++i)
                    for (int comp = 0; comp < 3; ++comp)
                        No[comp][cidx(B, c, i, j, k)] = conv_quick(g, bufs, comp, i, j, k, h);
    }
    free(gu); free(gv); free(gw);
}

int orc_set_scheme(orc_grid *g, int scheme, double cn_rtol, int cn_max) {
    if (scheme != 0 && scheme != 1) {
        snprintf(g_err, sizeof g_err, "unknown momentum scheme %d", scheme);
        return -1;
    }
    if (scheme == 0 && g->scheme == 1) g->ab2_restart = 1;
    g->scheme = scheme;
    g->cn_rtol = cn_rtol;
    g->cn_max = cn_max;
    return 0;
}

void orc_convection_diffusion(const orc_grid *g, const double *u, const double *v,
                              const double *w, const double *ub, double *nx, double *ny,
                              double *nz, double *lx, double *ly, double *lz) {
    int B = g->B;
    size_t G3 = (size_t)g->G * g->G * g->G;
    double *gu = (double *)malloc(sizeof(double) * G3 * g->n_cubes);
    double *gv = (double *)malloc(sizeof(double) * G3 * g->n_cubes);
    double *gw = (double *)malloc(sizeof(double) * G3 * g->n_cubes);
    orc_fill_ghosts(g, u, 0, ub, gu);
    orc_fill_ghosts(g, v, 1, ub, gv);
    orc_fill_ghosts(g, w, 2, ub, gw);
    double *No[3] = {nx, ny, nz}, *Lo[3] = {lx, ly, lz};
#pragma omp parallel for schedule(static)
    for (int c = 0; c < g->n_cubes; ++c) {
        double *bufs[3] = {gu + c * G3, gv + c * G3, gw + c * G3};
        double h = cell_h(g, c);
        for (int k = 0; k < B; ++k)
            for (int j = 0; j < B; ++j)
                for (int i = 0; i < B; ++i)
                    for (int comp = 0; comp < 3; ++comp)
                        conv_diff(g, bufs, comp, i, j, k, h, &No[comp][cidx(B, c, i, j, k)],
                                  &Lo[comp][cidx(B, c, i, j, k)]);
    }
    free(gu); free(gv); free(gw);
}

/* ------------------------------------------------------- pressure operator */

/* One face of cell (i,j,k) of cube c with outward normal face index fc: call back
 * each sub-face with (coefficient A_f/d_f, neighbour value or NAN for Dirichlet 0,
 * fraction of the face area).  Neumann faces produce no sub-face. */
typedef struct {
    int n;
    double coef[4], pn[4], frac[4];
    int dirichlet[4];
} subfaces;

static void face_subfaces(const orc_grid *g, const double *p, int c, int fc, int i, int j,
                          int k, subfaces *out) {
    int B = g->B, d = fc / 2, side = fc % 2, s = g->sim_of[c];
    int q[3] = {i, j, k};
    int a = q[tan1(d)], b = q[tan2(d)];
    double h = cell_h(g, c);
    out->n = 0;
    int at_face = side ? (q[d] == B - 1) : (q[d] == 0);
    if (!at_face) {
        int r[3] = {i, j, k};
        r[d] += side ? 1 : -1;
        out->n = 1;
        out->coef[0] = h; out->pn[0] = p[cidx(B, c, r[0], r[1], r[2])];
        out->frac[0] = 1.0; out->dirichlet[0] = 0;
        return;
    }
    int nb = g->nb[6 * c + fc];
    if (nb >= 0) {
        out->n = 1;
        out->coef[0] = h; out->pn[0] = fval(g, p, nb, d, side ? 0 : B - 1, a, b);
        out->frac[0] = 1.0; out->dirichlet[0] = 0;
    } else if (nb == NB_BOUNDARY) {
        if (g->bc[6 * s + fc] == BC_OUTFLOW) {
            out->n = 1;
            out->coef[0] = h; out->pn[0] = -p[cidx(B, c, i, j, k)];
            out->frac[0] = 1.0; out->dirichlet[0] = 1;
        }
    } else if (nb == NB_COARSE) { /* fine cell, one coarse neighbour: sub-face of area h^2 */
        int C = g->nb_coarse[6 * c + fc];
        int sf = cell_span(g, c), sc = cell_span(g, C);
        int A = (g->ijk[3 * c + tan1(d)] + a * sf - g->ijk[3 * C + tan1(d)]) / sc;
        int Bb = (g->ijk[3 * c + tan2(d)] + b * sf - g->ijk[3 * C + tan2(d)]) / sc;
        out->n = 1;
        out->coef[0] = h * h / (1.5 * h); out->pn[0] = fval(g, p, C, d, side ? 0 : B - 1, A, Bb);
        out->frac[0] = 1.0; out->dirichlet[0] = 0;
    } else { /* coarse cell, four fine neighbours each with a sub-face of area (h/2)^2 */
        int qa = (2 * a) / B, qb = (2 * b) / B;
        int F = g->nb_fine[(6 * c + fc) * 4 + qb * 2 + qa];
        int fa = 2 * a - qa * B, fb = 2 * b - qb * B;
        double hf = 0.5 * h;
        for (int bb = 0; bb < 2; ++bb)
            for (int aa = 0; aa < 2; ++aa) {
                int m = out->n++;
                out->coef[m] = hf * hf / (0.75 * h);
                out->pn[m] = fval(g, p, F, d, side ? 0 : B - 1, fa + aa, fb + bb);
                out->frac[m] = 0.25;
                out->dirichlet[m] = 0;
            }
    }
}

static void apply_range(const orc_grid *g, const double *x, double *y, int c0, int c1) {
    int B = g->B;
#pragma omp parallel for schedule(static)
    for (int c = c0; c < c1; ++c)
        for (int k = 0; k < B; ++k)
            for (int j = 0; j < B; ++j)
                for (int i = 0; i < B; ++i) {
                    double xi = x[cidx(B, c, i, j, k)], acc = 0.0;
                    for (int fc = 0; fc < 6; ++fc) {
                        subfaces sf;
                        face_subfaces(g, x, c, fc, i, j, k, &sf);
                        for (int m = 0; m < sf.n; ++m) acc += sf.coef[m] * (xi - sf.pn[m]);
                    }
                    y[cidx(B, c, i, j, k)] = acc;
                }
}

void orc_apply_poisson(const orc_grid *g, const double *x, double *y) {
    apply_range(g, x, y, 0, g->n_cubes);
}

void orc_poisson_diag(const orc_grid *g, double *dg) {
    int B = g->B;
    size_t n = (size_t)g->n_cubes * B * B * B;
    double *one = (double *)malloc(sizeof(double) * n);
    for (size_t q = 0; q < n; ++q) one[q] = 0.0;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < g->n_cubes; ++c)
        for (int k = 0; k < B; ++k)
            for (int j = 0; j < B; ++j)
                for (int i = 0; i < B; ++i) {
                    double acc = 0.0;
                    for (int fc = 0; fc < 6; ++fc) {
                        subfaces sf;
                        face_subfaces(g, one, c, fc, i, j, k, &sf);
                        for (int m = 0; m < sf.n; ++m) acc += sf.coef[m] * (sf.dirichlet[m] ? 2.0 : 1.0);
                    }
                    dg[cidx(B, c, i, j, k)] = acc;
                }
    free(one);
}

/* ---------------------------------------------------------- face velocities */

/* Normal velocity through each sub-face of face fc of cell (i,j,k): interior faces
 * average the two cell values (R2), 2:1 faces interpolate linearly between the
 * fine and the coarse centre, domain faces take the boundary value (outflow: ubn). */
static void face_normal_velocity(const orc_grid *g, const double *un, const double *ubn,
                                 int c, int fc, int i, int j, int k, int *nsub,
                                 double U[4], double frac[4]) {
    int B = g->B, d = fc / 2, side = fc % 2, s = g->sim_of[c];
    int q[3] = {i, j, k};
    int a = q[tan1(d)], b = q[tan2(d)];
    double u0 = un[cidx(B, c, i, j, k)];
    int at_face = side ? (q[d] == B - 1) : (q[d] == 0);
    *nsub = 1;
    frac[0] = 1.0;
    if (!at_face) {
        int r[3] = {i, j, k};
        r[d] += side ? 1 : -1;
        U[0] = 0.5 * (u0 + un[cidx(B, c, r[0], r[1], r[2])]);
        return;
    }
    int nb = g->nb[6 * c + fc];
    if (nb >= 0) {
        U[0] = 0.5 * (u0 + fval(g, un, nb, d, side ? 0 : B - 1, a, b));
    } else if (nb == NB_BOUNDARY) {
        int bcf = g->bc[6 * s + fc];
        if (bcf == BC_SLIP) U[0] = 0.0;
        else if (bcf == BC_OUTFLOW)
            U[0] = ubn[(((size_t)g->slot[6 * c + fc] * 3 + d) * B + b) * B + a];
        else U[0] = face_velocity(g, c, fc, d, a, b);
    } else if (nb == NB_COARSE) {
        int C = g->nb_coarse[6 * c + fc];
        int sf = cell_span(g, c), sc = cell_span(g, C);
        int A = (g->ijk[3 * c + tan1(d)] + a * sf - g->ijk[3 * C + tan1(d)]) / sc;
        int Bb = (g->ijk[3 * c + tan2(d)] + b * sf - g->ijk[3 * C + tan2(d)]) / sc;
        double uc = fval(g, un, C, d, side ? 0 : B - 1, A, Bb);
        U[0] = (2.0 * u0 + uc) / 3.0;
    } else {
        int qa = (2 * a) / B, qb = (2 * b) / B;
        int F = g->nb_fine[(6 * c + fc) * 4 + qb * 2 + qa];
        int fa = 2 * a - qa * B, fb = 2 * b - qb * B;
        *nsub = 4;
        for (int bb = 0; bb < 2; ++bb)
            for (int aa = 0; aa < 2; ++aa) {
                double uf = fval(g, un, F, d, side ? 0 : B - 1, fa + aa, fb + bb);
                U[bb * 2 + aa] = (2.0 * uf + u0) / 3.0;
                frac[bb * 2 + aa] = 0.25;
            }
    }
}

void orc_rhs(const orc_grid *g, const double *us, const double *vs, const double *ws,
             const double *ub_new, double *b) {
    int B = g->B;
    const double *comp[3] = {us, vs, ws};
#pragma omp parallel for schedule(static)
    for (int c = 0; c < g->n_cubes; ++c) {
        double h = cell_h(g, c), dt = g->dt[g->sim_of[c]];
        for (int k = 0; k < B; ++k)
            for (int j = 0; j < B; ++j)
                for (int i = 0; i < B; ++i) {
                    double div = 0.0; /* (1/V) sum A_f U_f.n with A_f = frac * h^2 */
                    for (int fc = 0; fc < 6; ++fc) {
                        int ns;
                        double U[4], fr[4];
                        face_normal_velocity(g, comp[fc / 2], ub_new, c, fc, i, j, k, &ns, U, fr);
                        double sum = 0.0;
                        for (int m = 0; m < ns; ++m) sum += fr[m] * U[m];
                        div += (fc % 2) ? sum : -sum;
                    }
                    b[cidx(B, c, i, j, k)] = div / (h * dt); /* rho = 1 */
                }
    }
}

/* ------------------------------------------------------------------- PCG */

static double sim_dot(const orc_grid *g, int s, const double *x, const double *y,
                      double *part) {
    int B3 = g->B * g->B * g->B;
    int c0 = g->sim_off[s], c1 = g->sim_off[s + 1];
#pragma omp parallel for schedule(static)
    for (int c = c0; c < c1; ++c) {
        double acc = 0.0;
        for (int q = 0; q < B3; ++q) acc += x[(size_t)c * B3 + q] * y[(size_t)c * B3 + q];
        part[c] = acc;
    }
    double tot = 0.0;
    for (int c = c0; c < c1; ++c) tot += part[c];
    return tot;
}

static int sim_all_neumann(const orc_grid *g, int s) {
    for (int f = 0; f < 6; ++f)
        if (g->bc[6 * s + f] == BC_OUTFLOW) return 0;
    return 1;
}

int orc_solve_pressure(const orc_grid *g, const double *b, double *p, double rtol,
                       int max_iter, orc_stats *stats) {
    int B = g->B, B3 = B * B * B, status = 0;
    size_t n = (size_t)g->n_cubes * B3;
    double *rhs = (double *)malloc(sizeof(double) * n), *r = (double *)malloc(sizeof(double) * n);
    double *z = (double *)malloc(sizeof(double) * n), *pd = (double *)malloc(sizeof(double) * n);
    double *q = (double *)malloc(sizeof(double) * n), *dg = (double *)malloc(sizeof(double) * n);
    double *part = (double *)malloc(sizeof(double) * (g->n_cubes + 1));
    orc_poisson_diag(g, dg);
    /* rhs = -V b; for all-Neumann sims the volume mean of b is removed first (R10) */
    for (int s = 0; s < g->n_sims; ++s) {
        double mean = 0.0;
        if (sim_all_neumann(g, s)) {
            double vb = 0.0, vol = 0.0;
            for (int c = g->sim_off[s]; c < g->sim_off[s + 1]; ++c) {
                double V = pow(cell_h(g, c), 3), acc = 0.0;
                for (int t = 0; t < B3; ++t) acc += b[(size_t)c * B3 + t];
                vb += V * acc;
                vol += V * B3;
            }
            mean = vb / vol;
        }
        for (int c = g->sim_off[s]; c < g->sim_off[s + 1]; ++c) {
            double V = pow(cell_h(g, c), 3);
            for (int t = 0; t < B3; ++t)
                rhs[(size_t)c * B3 + t] = -V * (b[(size_t)c * B3 + t] - mean);
        }
    }
    orc_apply_poisson(g, p, q);
    for (size_t t = 0; t < n; ++t) {
        r[t] = rhs[t] - q[t];
        z[t] = r[t] / dg[t];
        pd[t] = z[t];
    }
    /* every sim runs its own CG on its own cubes; the operator never couples sims */
    for (int s = 0; s < g->n_sims; ++s) {
        size_t lo = (size_t)g->sim_off[s] * B3, hi = (size_t)g->sim_off[s + 1] * B3;
        double bn = sqrt(sim_dot(g, s, rhs, rhs, part));
        if (bn == 0.0) { /* b = 0: the solution is p = 0 */
            for (size_t t = lo; t < hi; ++t) p[t] = 0.0;
            if (stats) { stats[s].cg_iters = 0; stats[s].rel_resid = 0.0; }
            continue;
        }
        double rr = sim_dot(g, s, r, r, part);
        double rz = sim_dot(g, s, r, z, part);
        int it = 0;
        while (sqrt(rr) > rtol * bn && it < max_iter) {
            apply_range(g, pd, q, g->sim_off[s], g->sim_off[s + 1]); /* K never couples sims */
            double alpha = rz / sim_dot(g, s, pd, q, part);
            for (size_t t = lo; t < hi; ++t) {
                p[t] += alpha * pd[t];
                r[t] -= alpha * q[t];
                z[t] = r[t] / dg[t];
            }
            double rz_new = sim_dot(g, s, r, z, part);
            rr = sim_dot(g, s, r, r, part);
            double beta = rz_new / rz;
            rz = rz_new;
            for (size_t t = lo; t < hi; ++t) pd[t] = z[t] + beta * pd[t];
            ++it;
        }
        if (stats) {
            stats[s].cg_iters = it;
            stats[s].rel_resid = bn > 0.0 ? sqrt(rr) / bn : 0.0;
        }
        if (bn > 0.0 && sqrt(rr) > rtol * bn) status = -3;
    }
    free(rhs); free(r); free(z); free(pd); free(q); free(dg); free(part);
    return status;
}

/* ----------------------------------------------------------------- the step */

/* face gradient of p through face fc of cell (i,j,k), area-weighted over sub-faces */
static double face_gradient(const orc_grid *g, const double *p, int c, int fc, int i, int j,
                            int k) {
    subfaces sf;
    face_subfaces(g, p, c, fc, i, j, k, &sf);
    double h = cell_h(g, c), pi = p[cidx(g->B, c, i, j, k)], G = 0.0;
    for (int m = 0; m < sf.n; ++m) {
        double dist = sf.coef[m] > 0 ? (sf.frac[m] * h * h) / sf.coef[m] : 1.0; /* d_f = A_f / coef */
        double sub = (sf.pn[m] - pi) / dist;
        G += sf.frac[m] * sub;
    }
    return (fc % 2) ? G : -G; /* gradient along +axis */
}

/* Lagrangian particles of a step (R19); NULL in orc_step (solid fraction). */
typedef struct {
    int n;
    double *X;
    const int32_t *sim, *body;
    const double *dV;
    double *F; /* [n*3] force per particle of the last step, may be NULL */
} particle_args;

static int step_impl(const orc_grid *g, double *u, double *v, double *w, double *p, double *nx,
                     double *ny, double *nz, double *ub, int32_t *step, int nsteps, double rtol,
                     int max_iter, orc_stats *stats, const particle_args *P) {
    int B = g->B, B3 = B * B * B, status = 0;
    size_t n = (size_t)g->n_cubes * B3, G3 = (size_t)g->G * g->G * g->G;
    size_t nub = (size_t)g->n_slots * 3 * B * B;
    double *us = (double *)malloc(sizeof(double) * n), *vs = (double *)malloc(sizeof(double) * n);
    double *ws = (double *)malloc(sizeof(double) * n), *b = (double *)malloc(sizeof(double) * n);
    double *phi = (double *)malloc(sizeof(double) * n);
    double *bu = (double *)malloc(sizeof(double) * n), *bv = (double *)malloc(sizeof(double) * n);
    double *bw = (double *)malloc(sizeof(double) * n);
    double *gu = (double *)malloc(sizeof(double) * G3 * g->n_cubes);
    double *gv = (double *)malloc(sizeof(double) * G3 * g->n_cubes);
    double *gw = (double *)malloc(sizeof(double) * G3 * g->n_cubes);
    double *ubn = (double *)malloc(sizeof(double) * (nub + 1));
    double *drag = (double *)malloc(sizeof(double) * 3 * (g->n_cubes + 1));
    double *tt = (double *)malloc(sizeof(double) * (g->n_sims + 1));
    orc_stats *st = (orc_stats *)calloc(g->n_sims + 1, sizeof(orc_stats));
    double *vel[3] = {u, v, w}, *vstar[3] = {us, vs, ws}, *Nl[3] = {nx, ny, nz};
    int np = P ? P->n : 0;
    double *pU = (double *)malloc(sizeof(double) * (3 * (size_t)np + 1));
    double *pF = (double *)malloc(sizeof(double) * (3 * (size_t)np + 1));
    double *pS = (double *)malloc(sizeof(double) * ((size_t)np + 1));
    double *pdrag = (double *)calloc(3 * (size_t)g->n_sims + 1, sizeof(double));
    int cn = g->scheme == 1;
    double *cnbuf = (double *)malloc(sizeof(double) * (cn ? 9 * n : 1));
    double *cnE[3], *cnA[3], *cnB[3];
    for (int e = 0; e < 3; ++e) {
        cnE[e] = cnbuf + (cn ? (size_t)e * n : 0);
        cnA[e] = cnbuf + (cn ? (size_t)(3 + e) * n : 0);
        cnB[e] = cnbuf + (cn ? (size_t)(6 + e) * n : 0);
    }
    double *cnpart = (double *)malloc(sizeof(double) * (2 * (size_t)g->n_cubes + 1));
    int *cndone = (int *)calloc((size_t)g->n_sims + 1, sizeof(int));
    double *cnprev = (double *)calloc((size_t)g->n_sims + 1, sizeof(double));

    for (int it = 0; it < nsteps; ++it) {
        /* (a) body geometry and velocity at t^n (particles: no solid fraction) */
        for (int s = 0; s < g->n_sims; ++s) tt[s] = step[s] * g->dt[s];
        if (P) {
            for (size_t q = 0; q < n; ++q) phi[q] = bu[q] = bv[q] = bw[q] = 0.0;
        } else {
            orc_solid_fraction(g, tt, phi, bu, bv, bw);
        }
        /* (b) halo of u^n (outflow ghosts from u_b^n) */
        orc_fill_ghosts(g, u, 0, ub, gu);
        orc_fill_ghosts(g, v, 1, ub, gv);
        orc_fill_ghosts(g, w, 2, ub, gw);
        /* (d) outflow face values u_b^{n+1} (R8) */
        for (int c = 0; c < g->n_cubes; ++c)
            for (int fc = 0; fc < 6; ++fc) {
                int sl = g->slot[6 * c + fc];
                if (sl < 0) continue;
                int s = g->sim_of[c], d = fc / 2, side = fc % 2;
                double h = cell_h(g, c), dt = g->dt[s], Uc = g->uconv[s];
                for (int comp = 0; comp < 3; ++comp)
                    for (int bb = 0; bb < B; ++bb)
                        for (int aa = 0; aa < B; ++aa) {
                            size_t id = (((size_t)sl * 3 + comp) * B + bb) * B + aa;
                            double u0 = fval(g, vel[comp], c, d, side ? B - 1 : 0, aa, bb);
                            ubn[id] = ub[id] - Uc * dt * (ub[id] - u0) / (0.5 * h);
                        }
            }
        /* (c') QUICK + Crank-Nicolson (R20): explicit half E (ghosts of u^n with the
         * outflow values of t^n), the iteration for u~ (ghosts of the iterates, velocities
         * of t^{n+1}, with the outflow values of t^{n+1} from (d)), then the IB forcing */
        if (g->scheme == 1) {
#pragma omp parallel for schedule(static)
            for (int c = 0; c < g->n_cubes; ++c) {
                int s = g->sim_of[c];
                double h = cell_h(g, c), dt = g->dt[s], nu = g->nu[s];
                double *bufs[3] = {gu + c * G3, gv + c * G3, gw + c * G3};
                for (int k = 0; k < B; ++k)
                    for (int j = 0; j < B; ++j)
                        for (int i = 0; i < B; ++i)
                            for (int comp = 0; comp < 3; ++comp) {
                                double Nc, L, N;
                                conv_diff(g, bufs, comp, i, j, k, h, &Nc, &L);
                                N = conv_quick(g, bufs, comp, i, j, k, h);
                                size_t id = cidx(B, c, i, j, k);
                                cnE[comp][id] = vel[comp][id] + dt * (-0.5 * N + 0.5 * nu * L);
                                cnA[comp][id] = 2.0 * cnE[comp][id] - vel[comp][id];
                            }
            }
            for (int s = 0; s < g->n_sims; ++s) {
                cndone[s] = 0;
                cnprev[s] = 0.0;
            }
            for (int kk = 0; kk < g->cn_max; ++kk) {
                int alive = 0;
                for (int s = 0; s < g->n_sims; ++s) alive |= !cndone[s];
                if (!alive) break;
                orc_fill_ghosts(g, cnA[0], 0, ubn, gu);
                orc_fill_ghosts(g, cnA[1], 1, ubn, gv);
                orc_fill_ghosts(g, cnA[2], 2, ubn, gw);
#pragma omp parallel for schedule(static)
                for (int c = 0; c < g->n_cubes; ++c) {
                    int s = g->sim_of[c];
                    double h = cell_h(g, c), dt = g->dt[s], nu = g->nu[s];
                    double *bufs[3] = {gu + c * G3, gv + c * G3, gw + c * G3};
                    double den = 1.0 + 3.0 * dt * nu / (h * h), d2 = 0.0, u2 = 0.0;
                    for (int k = 0; k < B; ++k)
                        for (int j = 0; j < B; ++j)
                            for (int i = 0; i < B; ++i)
                                for (int comp = 0; comp < 3; ++comp) {
                                    size_t id = cidx(B, c, i, j, k);
                                    if (cndone[s]) {
                                        cnB[comp][id] = cnA[comp][id];
                                        continue;
                                    }
                                    const double *uc = bufs[comp];
                                    double N = conv_quick(g, bufs, comp, i, j, k, h), sn = 0.0;
                                    for (int d = 0; d < 3; ++d) {
                                        int p1[3] = {i, j, k}, m1[3] = {i, j, k};
                                        p1[d] += 1;
                                        m1[d] -= 1;
                                        sn += uc[gidx(g, p1[0], p1[1], p1[2])] +
                                              uc[gidx(g, m1[0], m1[1], m1[2])];
                                    }
                                    double un = (cnE[comp][id] - 0.5 * dt * N +
                                                 0.5 * dt * nu * sn / (h * h)) / den;
                                    double dd = un - cnA[comp][id];
                                    d2 += dd * dd;
                                    u2 += un * un;
                                    cnB[comp][id] = un;
                                }
                    cnpart[2 * c] = d2;
                    cnpart[2 * c + 1] = u2;
                }
                for (int s = 0; s < g->n_sims; ++s) {
                    if (cndone[s]) continue;
                    double d2 = 0.0, u2 = 0.0;
                    for (int c = g->sim_off[s]; c < g->sim_off[s + 1]; ++c) {
                        d2 += cnpart[2 * c];
                        u2 += cnpart[2 * c + 1];
                    }
                    const double fl = 64.0 * 0x1p-53;  /* 64 unit roundoffs of FP64 */
                    if (d2 <= g->cn_rtol * g->cn_rtol * u2 ||
                        (kk >= 1 && d2 <= fl * fl * u2 && d2 >= 0.99 * cnprev[s]))
                        cndone[s] = 1;
                    cnprev[s] = d2;
                }
                for (int comp = 0; comp < 3; ++comp) {
                    double *tmp = cnA[comp];
                    cnA[comp] = cnB[comp];
                    cnB[comp] = tmp;
                }
            }
#pragma omp parallel for schedule(static)
            for (int c = 0; c < g->n_cubes; ++c) {
                int s = g->sim_of[c];
                double h = cell_h(g, c), dt = g->dt[s], V = h * h * h;
                double fx = 0, fy = 0, fz = 0;
                const double *usb[3] = {bu, bv, bw};
                for (int k = 0; k < B; ++k)
                    for (int j = 0; j < B; ++j)
                        for (int i = 0; i < B; ++i) {
                            size_t id = cidx(B, c, i, j, k);
                            for (int comp = 0; comp < 3; ++comp) {
                                double ut = cnA[comp][id];
                                double du = phi[id] * (usb[comp][id] - ut);
                                vstar[comp][id] = ut + du;
                                double f = du / dt;
                                if (comp == 0) fx += f * V;
                                else if (comp == 1) fy += f * V;
                                else fz += f * V;
                            }
                        }
                drag[3 * c] = -fx; drag[3 * c + 1] = -fy; drag[3 * c + 2] = -fz;
            }
        } else {
        /* (c) momentum sub-step (R3) and IB forcing (R5) */
#pragma omp parallel for schedule(static)
        for (int c = 0; c < g->n_cubes; ++c) {
            int s = g->sim_of[c];
            double h = cell_h(g, c), dt = g->dt[s], nu = g->nu[s], V = h * h * h;
            double *bufs[3] = {gu + c * G3, gv + c * G3, gw + c * G3};
            double fx = 0, fy = 0, fz = 0;
            const double *usb[3] = {bu, bv, bw};
            for (int k = 0; k < B; ++k)
                for (int j = 0; j < B; ++j)
                    for (int i = 0; i < B; ++i) {
                        size_t id = cidx(B, c, i, j, k);
                        for (int comp = 0; comp < 3; ++comp) {
                            double N, L;
                            conv_diff(g, bufs, comp, i, j, k, h, &N, &L);
                            double Nprev = (step[s] == 0 || g->ab2_restart) ? N : Nl[comp][id];
                            double ut = vel[comp][id] + dt * (-(1.5 * N - 0.5 * Nprev) + nu * L);
                            double du = phi[id] * (usb[comp][id] - ut);
                            vstar[comp][id] = ut + du;
                            Nl[comp][id] = N;
                            double f = du / dt; /* force density on the fluid, rho = 1 */
                            if (comp == 0) fx += f * V;
                            else if (comp == 1) fy += f * V;
                            else fz += f * V;
                        }
                    }
            drag[3 * c] = -fx; drag[3 * c + 1] = -fy; drag[3 * c + 2] = -fz;
        }
        }
        /* (c') particles (R19): U = I[u~] at every particle, F = (U_s - U) / dt, then
         * u* = u~ + dt P[F]; the force on the body is -sum F dV */
        if (P) {
            for (int s = 0; s < 3 * g->n_sims; ++s) pdrag[s] = 0.0;
            for (int comp = 0; comp < 3; ++comp)
                orc_ib_interpolate(g, vstar[comp], np, P->X, P->sim, pU + (size_t)comp * np);
            for (int q = 0; q < np; ++q) {
                int s = P->sim[q];
                double Us[3];
                particle_body_velocity(g, s, P->body[q], P->X + 3 * q, tt[s], Us);
                for (int comp = 0; comp < 3; ++comp) {
                    double F = (Us[comp] - pU[(size_t)comp * np + q]) / g->dt[s];
                    pF[(size_t)comp * np + q] = F;
                    pdrag[3 * s + comp] -= F * P->dV[q];
                    if (P->F) P->F[3 * q + comp] = F;
                }
            }
            for (int comp = 0; comp < 3; ++comp) {
                for (int q = 0; q < np; ++q) pS[q] = g->dt[P->sim[q]] * pF[(size_t)comp * np + q];
                orc_ib_spread(g, np, P->X, P->sim, pS, P->dV, vstar[comp]);
            }
        }
        /* (e) Poisson right-hand side from u* and the new outflow values */
        orc_rhs(g, us, vs, ws, ubn, b);
        /* (f) pressure solve */
        int rc = orc_solve_pressure(g, b, p, rtol, max_iter, st);
        if (rc) status = rc;
        /* (g) projection (R1, R2): u = u* - dt * mean of the two face gradients */
#pragma omp parallel for schedule(static)
        for (int c = 0; c < g->n_cubes; ++c) {
            double dt = g->dt[g->sim_of[c]];
            for (int k = 0; k < B; ++k)
                for (int j = 0; j < B; ++j)
                    for (int i = 0; i < B; ++i) {
                        size_t id = cidx(B, c, i, j, k);
                        for (int d = 0; d < 3; ++d) {
                            double gm = face_gradient(g, p, c, 2 * d, i, j, k);
                            double gp = face_gradient(g, p, c, 2 * d + 1, i, j, k);
                            vel[d][id] = vstar[d][id] - dt * 0.5 * (gm + gp);
                        }
                    }
        }
        /* (h) diagnostics: divergence of corrected face velocities, drag, max |u| */
        for (int s = 0; s < g->n_sims; ++s) {
            double dn = 0.0, ds = 0.0, um = 0.0, F[3] = {0, 0, 0};
            for (int c = g->sim_off[s]; c < g->sim_off[s + 1]; ++c) {
                double h = cell_h(g, c), dt = g->dt[s];
                for (int e = 0; e < 3; ++e) F[e] += drag[3 * c + e];
                for (int k = 0; k < B; ++k)
                    for (int j = 0; j < B; ++j)
                        for (int i = 0; i < B; ++i) {
                            double dstar = 0.0, dnew = 0.0;
                            for (int fc = 0; fc < 6; ++fc) {
                                int ns;
                                double U[4], fr[4];
                                face_normal_velocity(g, vstar[fc / 2], ubn, c, fc, i, j, k, &ns, U, fr);
                                subfaces sf;
                                face_subfaces(g, p, c, fc, i, j, k, &sf);
                                double pi = p[cidx(B, c, i, j, k)];
                                double a1 = 0.0, a2 = 0.0;
                                for (int m = 0; m < ns; ++m) {
                                    double grad = 0.0; /* outward normal gradient of sub-face m */
                                    for (int mm = 0; mm < sf.n; ++mm)
                                        if (ns == sf.n && mm == m) {
                                            double dist = (sf.frac[mm] * h * h) / sf.coef[mm];
                                            grad = (sf.pn[mm] - pi) / dist;
                                        }
                                    double Un = (fc % 2) ? U[m] : -U[m];
                                    a1 += fr[m] * Un;
                                    a2 += fr[m] * (Un - dt * grad);
                                }
                                dstar += a1;
                                dnew += a2;
                            }
                            ds += (dstar / h) * (dstar / h);
                            dn += (dnew / h) * (dnew / h);
                            size_t id = cidx(B, c, i, j, k);
                            double m2 = sqrt(u[id] * u[id] + v[id] * v[id] + w[id] * w[id]);
                            if (m2 > um) um = m2;
                        }
            }
            if (P)
                for (int e = 0; e < 3; ++e) F[e] += pdrag[3 * s + e];
            if (stats) {
                stats[s].cg_iters = st[s].cg_iters;
                stats[s].rel_resid = st[s].rel_resid;
                stats[s].div_rel = ds > 0 ? sqrt(dn / ds) : 0.0;
                stats[s].drag[0] = F[0]; stats[s].drag[1] = F[1]; stats[s].drag[2] = F[2];
                stats[s].umax = um;
                stats[s].steps = step[s] + 1;
            }
            step[s] += 1;
        }
        memcpy(ub, ubn, sizeof(double) * nub);
        if (g->scheme == 0) ((orc_grid *)g)->ab2_restart = 0;
        /* (i) particles move with their body: X^{n+1} = X^n + dt U_s(X^n, t^{n+1}) */
        for (int q = 0; q < np; ++q) {
            int s = P->sim[q];
            double Us[3];
            particle_body_velocity(g, s, P->body[q], P->X + 3 * q, step[s] * g->dt[s], Us);
            for (int e = 0; e < 3; ++e) P->X[3 * q + e] += g->dt[s] * Us[e];
        }
    }
    free(us); free(vs); free(ws); free(b); free(phi); free(bu); free(bv); free(bw);
    free(gu); free(gv); free(gw); free(ubn); free(drag); free(tt); free(st);
    free(pU); free(pF); free(pS); free(pdrag);
    free(cnbuf); free(cnpart); free(cndone); free(cnprev);
    return status;
}

int orc_step(const orc_grid *g, double *u, double *v, double *w, double *p, double *nx,
             double *ny, double *nz, double *ub, int32_t *step, int nsteps, double rtol,
             int max_iter, orc_stats *stats) {
    return step_impl(g, u, v, w, p, nx, ny, nz, ub, step, nsteps, rtol, max_iter, stats, NULL);
}

int orc_step_particles(const orc_grid *g, double *u, double *v, double *w, double *p,
                       double *nx, double *ny, double *nz, double *ub, int32_t *step,
                       int nsteps, double rtol, int max_iter, orc_stats *stats, int n_particles,
                       double *X, const int32_t *psim, const int32_t *pbody, const double *dV,
                       double *F) {
    if (g->max_level != 0) {
        snprintf(g_err, sizeof g_err, "Lagrangian particles need a single-level grid");
        return -1;
    }
    particle_args P = {n_particles, X, psim, pbody, dV, F};
    return step_impl(g, u, v, w, p, nx, ny, nz, ub, step, nsteps, rtol, max_iter, stats, &P);
}

/* ------------------------------------------------- wavelet compression (R21) */

/* one CDF 5/3 lifting step on x[0 .. m) with stride st (m even >= 2); tmp holds m values */
static void lift53_forward(double *x, int m, int st, double *tmp) {
    int h = m / 2;
    for (int i = 0; i < h; ++i) { /* predict */
        double right = (2 * i + 2 < m) ? x[(2 * i + 2) * st] : x[(2 * i) * st];
        double t = x[(2 * i) * st] + right;
        t = 0.5 * t;
        tmp[h + i] = x[(2 * i + 1) * st] - t;
    }
    for (int i = 0; i < h; ++i) { /* update */
        double dl = i > 0 ? tmp[h + i - 1] : tmp[h];
        double t = dl + tmp[h + i];
        t = 0.25 * t;
        tmp[i] = x[(2 * i) * st] + t;
    }
    for (int i = 0; i < m; ++i) x[i * st] = tmp[i];
}

static void lift53_inverse(double *x, int m, int st, double *tmp) {
    int h = m / 2;
    for (int i = 0; i < h; ++i) { /* undo the update */
        double dl = i > 0 ? x[(h + i - 1) * st] : x[h * st];
        double t = dl + x[(h + i) * st];
        t = 0.25 * t;
        tmp[2 * i] = x[i * st] - t;
    }
    for (int i = 0; i < h; ++i) { /* undo the predict */
        double right = (2 * i + 2 < m) ? tmp[2 * i + 2] : tmp[2 * i];
        double t = tmp[2 * i] + right;
        t = 0.5 * t;
        tmp[2 * i + 1] = x[(h + i) * st] + t;
    }
    for (int i = 0; i < m; ++i) x[i * st] = tmp[i];
}

/* start of line (a, b) along axis d of a cube of edge B, and its stride */
static int line_base(int B, int d, int a, int b) {
    return d == 0 ? (b * B + a) * B : (d == 1 ? b * B * B + a : b * B + a);
}
static int line_stride(int B, int d) { return d == 0 ? 1 : (d == 1 ? B : B * B); }

/* forward / inverse transform of one cube of B^3 values in place (index (k B + j) B + i) */
void orc_dwt3_forward(int B, double *x) {
    double tmp[64];
    for (int m = B; m >= 2; m /= 2)
        for (int d = 0; d < 3; ++d)
            for (int b = 0; b < m; ++b)
                for (int a = 0; a < m; ++a)
                    lift53_forward(x + line_base(B, d, a, b), m, line_stride(B, d), tmp);
}

void orc_dwt3_inverse(int B, double *x) {
    double tmp[64];
    for (int m = 2; m <= B; m *= 2)
        for (int d = 2; d >= 0; --d)
            for (int b = 0; b < m; ++b)
                for (int a = 0; a < m; ++a)
                    lift53_inverse(x + line_base(B, d, a, b), m, line_stride(B, d), tmp);
}

static uint32_t zigzag(int32_t q) { return ((uint32_t)q << 1) ^ (uint32_t)(q >> 31); }
static int32_t unzigzag(uint32_t z) { return (int32_t)(z >> 1) ^ -(int32_t)(z & 1u); }

static void put_bit(uint32_t *w, uint64_t pos, int bit) {
    if (bit) w[pos >> 5] |= 1u << (pos & 31);
}
static int get_bit(const uint32_t *w, uint64_t pos) { return (w[pos >> 5] >> (pos & 31)) & 1u; }

/* Compress n_cubes cubes of B^3 values (cube-major) into out (capacity words).
 * Returns the number of words written, or -1 when the capacity is too small or a code
 * does not fit in 31 bits. */
long orc_wavelet_compress(int B, int n_cubes, const double *f, double step, uint32_t *out,
                          long capacity) {
    long B3 = (long)B * B * B, head = 8 + (long)n_cubes;
    if (capacity < head) return -1;
    memset(out, 0, sizeof(uint32_t) * (size_t)capacity);
    out[0] = 0x57434d42u; /* "BCMW" */
    out[1] = 1;
    out[2] = (uint32_t)B;
    out[3] = (uint32_t)n_cubes;
    memcpy(out + 6, &step, sizeof(double));
    double *x = (double *)malloc(sizeof(double) * (size_t)B3);
    uint32_t *z = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)B3);
    long pos = head;
    for (int c = 0; c < n_cubes; ++c) {
        memcpy(x, f + (size_t)c * B3, sizeof(double) * (size_t)B3);
        orc_dwt3_forward(B, x);
        uint64_t sum = 0;
        for (long q = 0; q < B3; ++q) {
            double r = nearbyint(x[q] / step);
            if (!(fabs(r) < 1073741824.0)) { free(x); free(z); return -1; }
            z[q] = zigzag((int32_t)r);
            sum += z[q];
        }
        uint64_t mean = sum / (uint64_t)B3;
        int k = 0;
        while (k < 24 && (mean >> (k + 1)) != 0) ++k;
        uint64_t nbits = 0;
        for (long q = 0; q < B3; ++q) {
            uint32_t u = z[q] >> k;
            nbits += u < 16 ? (uint64_t)u + 1 + k : 48;
        }
        long words = 1 + (long)((nbits + 31) / 32);
        if (pos + words > capacity) { free(x); free(z); return -1; }
        out[pos] = (uint32_t)k | (uint32_t)(nbits << 5);
        uint32_t *w = out + pos + 1;
        uint64_t b = 0;
        for (long q = 0; q < B3; ++q) {
            uint32_t u = z[q] >> k;
            if (u < 16) {
                for (uint32_t e = 0; e < u; ++e) put_bit(w, b++, 1);
                put_bit(w, b++, 0);
                for (int e = 0; e < k; ++e) put_bit(w, b++, (z[q] >> e) & 1u);
            } else {
                for (int e = 0; e < 16; ++e) put_bit(w, b++, 1);
                for (int e = 0; e < 32; ++e) put_bit(w, b++, (z[q] >> e) & 1u);
            }
        }
        out[8 + c] = (uint32_t)words;
        pos += words;
    }
    free(x);
    free(z);
    return pos;
}

/* Decode a stream of orc_wavelet_compress into f (n_cubes * B^3 values).  Returns 0, or
 * -1 on a malformed stream. */
int orc_wavelet_decompress(const uint32_t *in, long words, double *f) {
    if (words < 8 || in[0] != 0x57434d42u || in[1] != 1) return -1;
    int B = (int)in[2], n_cubes = (int)in[3];
    double step;
    memcpy(&step, in + 6, sizeof(double));
    long B3 = (long)B * B * B, pos = 8 + (long)n_cubes;
    if (words < pos) return -1;
    for (int c = 0; c < n_cubes; ++c) {
        long cw = (long)in[8 + c];
        if (cw < 1 || pos + cw > words) return -1;
        int k = (int)(in[pos] & 31u);
        uint64_t nbits = in[pos] >> 5;
        const uint32_t *w = in + pos + 1;
        uint64_t b = 0;
        double *x = f + (size_t)c * B3;
        for (long q = 0; q < B3; ++q) {
            uint32_t u = 0, z = 0;
            while (u < 16 && b < nbits && get_bit(w, b)) { ++u; ++b; }
            if (u < 16) {
                ++b; /* the zero */
                uint32_t r = 0;
                for (int e = 0; e < k; ++e) r |= (uint32_t)get_bit(w, b++) << e;
                z = (u << k) | r;
            } else {
                for (int e = 0; e < 32; ++e) z |= (uint32_t)get_bit(w, b++) << e;
            }
            if (b > nbits) return -1;
            x[q] = (double)unzigzag(z) * step;
        }
        orc_dwt3_inverse(B, x);
        pos += cw;
    }
    return 0;
}
